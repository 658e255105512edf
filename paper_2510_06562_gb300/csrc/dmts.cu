// C ABI of the DMTS library (declared in include/dmts.h).
//
// A context owns the device state (FP64 positions and velocities, the two
// models' FP32 parameters, neighbour lists and feature buffers), one CUDA
// stream and the CUDA graphs of the integration steps: one graph per
// (n_inner, dt) holds a whole outer step of Algorithm 1 -- n_inner times
// (kicks + drifts, small-model neighbour list and forces) followed by the
// big-model neighbour list and forces and the closing half-kick -- and is
// replayed once per outer step. Neighbour capacity overflow is detected on
// the device; the host restores the state saved at the start of the call,
// grows the capacity, re-captures the graph and runs the call again.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dmts.h"
#include "internal.cuh"
#include "umma.cuh"

namespace dmts {
thread_local long long* g_launch_counter = nullptr;

void smem_opt_in(const void* kern, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!done.insert({kern, dev}).second) return;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
        cudaGetLastError();                  // not sticky: a launch that needs more reports its own error
        done.erase({kern, dev});
    }
}
double accel_constant();
}  // namespace dmts

using namespace dmts;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? DMTS_ERR_OOM : DMTS_ERR_CUDA,  \
                        "%s: %s", #expr, cudaGetErrorString(e_));                        \
    } while (0)

// Context options: a flat JSON object whose values are numbers or booleans
// (true = 1, false = 0), e.g. {"skin": 1.0, "autotune": false}. The whole
// string is checked before any device work: malformed JSON, a key that is
// not an option, a repeated key, or another kind of value is an argument
// error, so a misspelt option cannot pass unnoticed.
constexpr const char* kOptionKeys[] = {
    "atom_tensor_cores", "atoms_per_cta_big", "atoms_per_cta_small", "autotune", "cell_capacity",
    "concurrent_models", "edge_capacity_factor", "fallback_threshold", "langevin_friction", "row_capacity",
    "seed", "skin", "temperature"};

struct Options {
    std::vector<std::pair<std::string, double>> kv;
    double get(const char* key, double dflt) const {
        for (const auto& e : kv)
            if (e.first == key) return e.second;
        return dflt;
    }
};

int parse_options(const char* js, Options& out) {
    out.kv.clear();
    if (!js) return DMTS_OK;
    const char* p = js;
    auto ws = [&p] { while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') ++p; };
    ws();
    if (!*p) return DMTS_OK;                                   // empty string: no options
    if (*p != '{') return fail(DMTS_ERR_ARG, "options: a JSON object was expected");
    ++p;
    ws();
    if (*p == '}') {
        ++p;
        ws();
        return *p ? fail(DMTS_ERR_ARG, "options: text after the closing brace") : DMTS_OK;
    }
    for (;;) {
        if (*p != '"') return fail(DMTS_ERR_ARG, "options: a quoted key was expected at offset %d", (int)(p - js));
        const char* k0 = ++p;
        while (*p && *p != '"' && *p != '\\') ++p;
        if (*p != '"') return fail(DMTS_ERR_ARG, "options: unterminated key or escape in a key");
        const std::string key(k0, p - k0);
        ++p;
        bool known = false;
        for (const char* k : kOptionKeys) known = known || key == k;
        if (!known) return fail(DMTS_ERR_ARG, "options: unknown key \"%s\"", key.c_str());
        for (const auto& e : out.kv)
            if (e.first == key) return fail(DMTS_ERR_ARG, "options: key \"%s\" repeated", key.c_str());
        ws();
        if (*p != ':') return fail(DMTS_ERR_ARG, "options: ':' expected after \"%s\"", key.c_str());
        ++p;
        ws();
        double v = 0.0;
        if (strncmp(p, "true", 4) == 0) {
            v = 1.0;
            p += 4;
        } else if (strncmp(p, "false", 5) == 0) {
            v = 0.0;
            p += 5;
        } else if (*p == '-' || (*p >= '0' && *p <= '9')) {
            char* end = nullptr;
            v = strtod(p, &end);
            if (end == p || !isfinite(v)) return fail(DMTS_ERR_ARG, "options: bad number for \"%s\"", key.c_str());
            p = end;
        } else {
            return fail(DMTS_ERR_ARG, "options: \"%s\" must be a number or a boolean", key.c_str());
        }
        out.kv.emplace_back(key, v);
        ws();
        if (*p == ',') {
            ++p;
            ws();
            continue;
        }
        if (*p != '}') return fail(DMTS_ERR_ARG, "options: ',' or '}' expected after \"%s\"", key.c_str());
        ++p;
        ws();
        return *p ? fail(DMTS_ERR_ARG, "options: text after the closing brace") : DMTS_OK;
    }
}

struct Model {
    bool present = false;
    int F = 0, K = 0, L = 0, S = 0, precision = 0;
    double rc = 0;
    double rep_a = 0, rep_rho = 1, rep_rc = 0;
    float* erep = nullptr;
    size_t n_params = 0;
    std::vector<double> hp;            // the parameters as last uploaded (FP64, flat order)
    ModelOffsets off{};
    float* P = nullptr;
    int nc = 0, n_cells = 0;
    int *cell_count = nullptr, *cell_start = nullptr, *cell_atoms = nullptr, *atom_cell = nullptr,
        *atom_slot = nullptr, *atom_pos = nullptr;
    uint4* cell_q = nullptr;
    int ccap = 0;                      // skin 0: slots per cell ([n_cells][ccap] cell_atoms / cell_q)
    bool placed = false;               // while capturing: the integrator kernel fills the cells
    int row_cap = 0;
    long long e_cap = 0;
    int *nbr_tmp = nullptr, *nbr_cnt = nullptr, *row_ptr = nullptr, *col = nullptr, *recv = nullptr;
    int *block_sum = nullptr, *chunk_sum = nullptr;   // folded row scan of fresh builds
    unsigned int* ticket = nullptr;
    int vl_cap = 0;                    // Verlet-skin candidate rows [N][vl_cap] (ascending j)
    int *vl_rows = nullptr, *vl_cnt = nullptr;
    float *h = nullptr, *gh = nullptr, *force = nullptr, *vir6 = nullptr;
    float* h0 = nullptr;               // [N][F] h^0 = A[Z_i] (constant between parameter uploads)
    float* PT = nullptr;               // transposed weight copies for the per-atom MLPs
    float* u[kMaxLayers] = {};
    float* z[kMaxLayers] = {};
    float* mbar[2] = {};
    unsigned char* um[kMaxLayers] = {};   // BF16 u^l | mbar^l rows for the tensor-core backward
    float* msg = nullptr;              // [N][F] per-atom sums between edge and atom kernels
    unsigned char* wt = nullptr;       // BF16 filter-weight operand tiles, per layer
    unsigned char* at = nullptr;       // BF16 hi/lo tiles of the per-atom MLP matrices (tensor-core path)
    size_t wt_layer_bytes = 0;
    double *Ei = nullptr, *E = nullptr, *W = nullptr;
    int apc_fwd = 16, apc_bwd = 16;    // FP32 kernels: atoms per CTA
    int cps_fwd = 0, cps_bwd = 0;      // tensor-core kernels: persistent CTAs per SM (0: as many as fit)
    int bwd_tiles = 0;                 // tensor-core backward: 128-pair tiles in flight per CTA (0: default)
    float* carry = nullptr;            // tensor-core path: per-tile partial sums of split rows
    SumScratch esum{};                 // scratch of the per-system energy sum
};

}  // namespace

struct dmts_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int N = 0, n_sys = 0;
    bool periodic = false;
    std::vector<int> h_off;
    std::vector<double> h_box;
    int *d_off = nullptr, *d_species = nullptr, *d_sys = nullptr;
    double *d_box = nullptr, *d_mass = nullptr, *d_inv_m = nullptr;
    double *d_x = nullptr, *d_v = nullptr;
    uint4* d_q = nullptr;
    Frame* d_frame = nullptr;
    double* d_stage = nullptr;   // [2][N*3]
    double *d_ke = nullptr, *d_ekin = nullptr;
    double* d_ring = nullptr;
    int ring_len = 0;
    double* d_epart = nullptr;             // fused energy epilogue: block partials
    unsigned int* d_eticket = nullptr;
    int* d_flags = nullptr;
    int* h_flags = nullptr;      // pinned
    double *d_bx = nullptr, *d_bv = nullptr;
    Model m[2];
    double rc_max = 0;
    // Verlet-skin lists shared by the two models: the model with the larger
    // cutoff (vl_src) builds candidate rows from its cell list at rc + skin,
    // the other filters its own from them; skin 0 rebuilds every evaluation.
    double skin = 0;
    double vl_thr2 = 0;                 // rebuild once max |x - x_ref|^2 exceeds this
    int vl_src = 1;
    double* d_xref = nullptr;           // FP64 SoA [3][N], positions of the last rebuild
    VerletState* d_vl = nullptr;
    // Langevin thermostat of Algorithm 1 (friction 0: NVE)
    double friction_ps = 0.0, temperature = 300.0;
    unsigned long long seed = 0;
    unsigned long long* d_rng = nullptr;   // [0] inner-step counter of the noise, [1] copy at call entry
    // force-difference monitor and single-time-step fallback (threshold 0: statistics only)
    double fb_threshold = 0.0;             // eV/A
    ForceMonitor* d_mon = nullptr;
    double *d_sx = nullptr, *d_sv = nullptr;   // state at the start of the outer step
    float* d_sf = nullptr;
    cudaStream_t aux = nullptr;            // captures the fallback body of the step graph
    // second stream of the step graph: the large-model evaluation at the end of
    // the outer step runs beside the last small-model evaluation (same positions)
    cudaStream_t s_big = nullptr;
    bool fold_small = false;           // while capturing a step: the integrator sums F_small's split rows
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool concurrent = true;
    SumScratch kesum{};                    // scratch of the per-system kinetic-energy sum
    bool atom_tc = true;                   // BF16 mode: per-atom MLPs on the tensor cores
    bool keep_msg = false;                 // every message row stays in memory (the distillation reads them)
    long long body_launches = 0, fallback_seen = 0;
    double cap_factor = 1.5;
    bool state_set = false, forces_valid = false;
    bool broken = false;
    bool autotune = true, tuned = false;
    // force-matching buffers (allocated on first use)
    float *fm_g = nullptr, *fm_m = nullptr, *fm_mdot = nullptr, *fm_mb = nullptr, *fm_mdb = nullptr,
          *fm_ubar = nullptr, *fm_pe = nullptr, *fm_pa = nullptr;
    double *fm_sq = nullptr, *fm_grad = nullptr, *fm_loss = nullptr, *fm_stage = nullptr;
    double *fm_eref = nullptr, *fm_ce = nullptr;   // reference energies [fm_eref_cap], dL/dE scratch
    int fm_eref_cap = 0;
    cudaGraphExec_t graph = nullptr;
    int g_n_inner = 0;
    double g_dt = 0;
    long long g_nodes = 0;
    long long launches = 0;
};

namespace {

struct LaunchScope {
    explicit LaunchScope(dmts_ctx* c) { g_launch_counter = &c->launches; }
    ~LaunchScope() { g_launch_counter = nullptr; }
};

// An NVTX range around a host-side call (named in profilers' timelines; NVTX
// is header-only and costs nothing unless a profiler is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T));
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

int check_model(const dmts_model_desc* d, const char* name) {
    if (!d) return fail(DMTS_ERR_ARG, "%s model descriptor is NULL", name);
    if (!(d->cutoff > 0)) return fail(DMTS_ERR_ARG, "%s model: cutoff must be > 0", name);
    if (d->n_feat != 32 && d->n_feat != 64) return fail(DMTS_ERR_ARG, "%s model: n_feat must be 32 or 64", name);
    if (d->n_radial < 1 || d->n_radial > 16) return fail(DMTS_ERR_ARG, "%s model: n_radial must be in [1, 16]", name);
    if (d->n_layers < 1 || d->n_layers > kMaxLayers) return fail(DMTS_ERR_ARG, "%s model: n_layers must be in [1, 4]", name);
    if (d->n_species < 1 || d->n_species > 16) return fail(DMTS_ERR_ARG, "%s model: n_species must be in [1, 16]", name);
    if (!d->params) return fail(DMTS_ERR_ARG, "%s model: params is NULL", name);
    ModelOffsets o = model_offsets(d->n_species, d->n_feat, d->n_radial, d->n_layers);
    if ((size_t)o.total != d->n_params)
        return fail(DMTS_ERR_ARG, "%s model: n_params = %zu, layout needs %d", name, d->n_params, o.total);
    if (d->precision != DMTS_FP32 && d->precision != DMTS_BF16_MLP)
        return fail(DMTS_ERR_ARG, "%s model: unknown precision %d", name, d->precision);
    for (size_t k = 0; k < d->n_params; ++k)
        if (!isfinite(d->params[k])) return fail(DMTS_ERR_ARG, "%s model: parameter %zu is not finite", name, k);
    if (!(d->rep_a >= 0) || !isfinite(d->rep_a)) return fail(DMTS_ERR_ARG, "%s model: rep_a must be >= 0", name);
    if (d->rep_a > 0 && (!(d->rep_rho > 0) || !(d->rep_cutoff > 0) || d->rep_cutoff > d->cutoff))
        return fail(DMTS_ERR_ARG, "%s model: need rep_rho > 0 and 0 < rep_cutoff <= cutoff", name);
    return DMTS_OK;
}

void free_model_nbr(Model& m) {
    dfree(m.nbr_tmp); dfree(m.col); dfree(m.recv); dfree(m.vl_rows); dfree(m.carry);
    m.nbr_tmp = m.col = m.recv = m.vl_rows = nullptr;
    m.carry = nullptr;
}

cudaError_t alloc_model_nbr(dmts_ctx* c, Model& m) {
    cudaError_t e;
    if ((e = dalloc(&m.nbr_tmp, (size_t)c->N * m.row_cap)) != cudaSuccess) return e;
    if ((e = dalloc(&m.col, (size_t)m.e_cap)) != cudaSuccess) return e;
    if ((e = dalloc(&m.recv, (size_t)m.e_cap)) != cudaSuccess) return e;
    if (c->skin > 0 && (e = dalloc(&m.vl_rows, (size_t)c->N * m.vl_cap)) != cudaSuccess) return e;
    const size_t tiles = (size_t)((m.e_cap + 127) / 128);
    if ((e = dalloc(&m.carry, tiles * 2 * (size_t)(m.F + 16))) != cudaSuccess) return e;
    return cudaSuccess;
}

void free_model(Model& m) {
    dfree(m.P);
    dfree(m.cell_count); dfree(m.cell_start); dfree(m.cell_atoms); dfree(m.atom_cell); dfree(m.atom_slot);
    dfree(m.atom_pos); dfree(m.cell_q);
    free_model_nbr(m);
    dfree(m.nbr_cnt); dfree(m.row_ptr); dfree(m.vl_cnt);
    dfree(m.block_sum); dfree(m.chunk_sum); dfree(m.ticket);
    dfree(m.h); dfree(m.gh); dfree(m.force); dfree(m.vir6); dfree(m.h0); dfree(m.PT);
    for (int l = 0; l < kMaxLayers; ++l) { dfree(m.u[l]); dfree(m.z[l]); dfree(m.um[l]); }
    dfree(m.mbar[0]); dfree(m.mbar[1]); dfree(m.esum.part); dfree(m.esum.ctr);
    dfree(m.Ei); dfree(m.E); dfree(m.W); dfree(m.erep); dfree(m.msg); dfree(m.wt); dfree(m.at);
    m = Model();
}

uint16_t bf16_bits(float x) {
    // round to nearest even (inputs are finite)
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// BF16 operand tiles of the filter weights of every layer, in the K-major
// tile layout the tensor-core kernels read: W1^T [F][16] (K zero-padded),
// W2^T [F][F] and W2 [F][F].
std::vector<uint16_t> build_weight_tiles(const Model& m, const std::vector<float>& pf) {
    const int F = m.F, K = m.K;
    const size_t per = m.wt_layer_bytes / 2;
    std::vector<uint16_t> t(per * m.L, 0);
    for (int l = 0; l < m.L; ++l) {
        uint16_t* b = t.data() + per * l;
        uint16_t* t1 = b;
        uint16_t* t2 = b + (size_t)F * 16;
        uint16_t* t3 = t2 + (size_t)F * F;
        const float* W1 = pf.data() + m.off.W1[l];
        const float* W2 = pf.data() + m.off.W2[l];
        for (int n = 0; n < F; ++n)
            for (int k = 0; k < 16; ++k)
                t1[umma::tile_offset(n, k, 16) / 2] = k < K ? bf16_bits(W1[k * F + n]) : 0;
        for (int n = 0; n < F; ++n)
            for (int k = 0; k < F; ++k) {
                t2[umma::tile_offset(n, k, F) / 2] = bf16_bits(W2[k * F + n]);
                t3[umma::tile_offset(n, k, F) / 2] = bf16_bits(W2[n * F + k]);
            }
    }
    return t;
}

float bf16_value(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float x;
    memcpy(&x, &u, 4);
    return x;
}

// Operand tiles of the per-atom MLP matrices for the tensor-core kernels
// (atom_tc.cu): per layer W_in, U1, U2 as B operands of X W (B[n][k] =
// W[k][n]) and of X W^T (B[n][k] = W[n][k]), then R1 both ways; each slot a
// high BF16 tile then the BF16 rounding of the remainder, K-major.
std::vector<uint16_t> build_atom_tiles(const Model& m, const std::vector<float>& pf) {
    const int F = m.F;
    const size_t FF = (size_t)F * F;
    std::vector<uint16_t> t((6 * (size_t)m.L + 2) * 2 * FF, 0);
    auto put = [&](size_t slot, int off, bool transpose) {
        uint16_t* hi = t.data() + slot * 2 * FF;
        uint16_t* lo = hi + FF;
        for (int n = 0; n < F; ++n)
            for (int k = 0; k < F; ++k) {
                const float w = transpose ? pf[off + (size_t)n * F + k] : pf[off + (size_t)k * F + n];
                const uint16_t h = bf16_bits(w);
                const size_t o = umma::tile_offset(n, k, F) / 2;
                hi[o] = h;
                lo[o] = bf16_bits(w - bf16_value(h));
            }
    };
    for (int l = 0; l < m.L; ++l) {
        put(6 * (size_t)l + 0, m.off.W_in[l], false);
        put(6 * (size_t)l + 1, m.off.U1[l], false);
        put(6 * (size_t)l + 2, m.off.U2[l], false);
        put(6 * (size_t)l + 3, m.off.W_in[l], true);
        put(6 * (size_t)l + 4, m.off.U1[l], true);
        put(6 * (size_t)l + 5, m.off.U2[l], true);
    }
    put(6 * (size_t)m.L, m.off.R1, false);
    put(6 * (size_t)m.L + 1, m.off.R1, true);
    return t;
}

// Transposed copies of the per-atom MLP matrices: W_in^T, U1^T, U2^T of each
// layer, then R1^T (each F x F, row-major).
std::vector<float> build_transposed(const Model& m, const std::vector<float>& pf) {
    const int F = m.F;
    const size_t FF = (size_t)F * F;
    std::vector<float> t((3 * (size_t)m.L + 1) * FF);
    auto put = [&](size_t slot, int off) {
        for (int r = 0; r < F; ++r)
            for (int k = 0; k < F; ++k) t[slot * FF + (size_t)k * F + r] = pf[off + (size_t)r * F + k];
    };
    for (int l = 0; l < m.L; ++l) {
        put(3 * l + 0, m.off.W_in[l]);
        put(3 * l + 1, m.off.U1[l]);
        put(3 * l + 2, m.off.U2[l]);
    }
    put(3 * (size_t)m.L, m.off.R1);
    return t;
}

int upload_params(dmts_ctx* c, Model& m, const double* params) {
    if (m.hp.data() != params) m.hp.assign(params, params + m.n_params);
    std::vector<float> pf(m.n_params);
    for (size_t k = 0; k < m.n_params; ++k) pf[k] = (float)params[k];
    CUDA_TRY(cudaMemcpyAsync(m.P, pf.data(), pf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    std::vector<uint16_t> tiles = build_weight_tiles(m, pf);
    CUDA_TRY(cudaMemcpyAsync(m.wt, tiles.data(), tiles.size() * 2, cudaMemcpyHostToDevice, c->stream));
    std::vector<float> tr = build_transposed(m, pf);
    CUDA_TRY(cudaMemcpyAsync(m.PT, tr.data(), tr.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    std::vector<uint16_t> at = build_atom_tiles(m, pf);
    CUDA_TRY(cudaMemcpyAsync(m.at, at.data(), at.size() * 2, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return DMTS_OK;
}

int init_model(dmts_ctx* c, Model& m, const dmts_model_desc* d, bool cells) {
    m.present = true;
    m.F = d->n_feat; m.K = d->n_radial; m.L = d->n_layers; m.S = d->n_species;
    m.precision = d->precision;
    m.rc = d->cutoff;
    m.rep_a = d->rep_a;
    m.rep_rho = d->rep_a > 0 ? d->rep_rho : 1.0;
    m.rep_rc = d->rep_a > 0 ? d->rep_cutoff : 0.0;
    m.n_params = d->n_params;
    m.off = model_offsets(m.S, m.F, m.K, m.L);
    const int N = c->N;
    CUDA_TRY(dalloc(&m.P, m.n_params));
    m.wt_layer_bytes = bf16_weight_tile_bytes(m.F);
    CUDA_TRY(dalloc(&m.wt, m.wt_layer_bytes * m.L));
    CUDA_TRY(dalloc(&m.PT, (3 * (size_t)m.L + 1) * m.F * m.F));
    CUDA_TRY(dalloc(&m.at, atom_tile_bytes(m.F, m.L)));
    int rc = upload_params(c, m, d->params);
    if (rc) return rc;
    // cells (periodic) and capacity estimates; with a skin the cells and the
    // candidate rows use rc + skin
    double expected;
    const double rv = m.rc + c->skin;
    if (c->periodic) {
        double L = c->h_box[0];
        int nc = (int)floor(L / (rv * (1.0 + 1e-9) + 1e-6));
        m.nc = (nc >= 3 && cells) ? nc : 0;
        double rho = (double)N / c->n_sys / (L * L * L);     // replicas of one box edge
        expected = 4.0 / 3.0 * M_PI * m.rc * m.rc * m.rc * rho;
        m.row_cap = std::min(N, (int)(ceil(expected * 1.5 / 32.0) * 32) + 32);
        m.e_cap = (long long)(N * expected * c->cap_factor) + 1024;
        const double expected_v = 4.0 / 3.0 * M_PI * rv * rv * rv * rho;
        m.vl_cap = std::min(N, (int)(ceil(expected_v * 1.5 / 32.0) * 32) + 32);
    } else {
        int mx = 0;
        long long sq = 0;
        for (int s = 0; s < c->n_sys; ++s) {
            int n = c->h_off[s + 1] - c->h_off[s];
            mx = std::max(mx, n);
            sq += (long long)n * (n - 1);
        }
        m.nc = 0;
        m.row_cap = std::max(32, ((mx + 31) / 32) * 32);
        m.vl_cap = m.row_cap;
        m.e_cap = std::max<long long>(1024, std::min<long long>(sq, (long long)(N * std::min(mx, 64) * c->cap_factor)) + 1024);
    }
    if (m.nc > 0) {
        m.n_cells = c->n_sys * m.nc * m.nc * m.nc;            // each system its own cells
        CUDA_TRY(dalloc(&m.cell_count, m.n_cells));
        CUDA_TRY(cudaMemset(m.cell_count, 0, sizeof(int) * m.n_cells));
        CUDA_TRY(dalloc(&m.atom_pos, N));
        if (c->skin > 0) {                 // compact cells rebuilt by count, scan and fill
            CUDA_TRY(dalloc(&m.cell_start, m.n_cells + 1));
            CUDA_TRY(dalloc(&m.atom_cell, N));
            CUDA_TRY(dalloc(&m.atom_slot, N));
            CUDA_TRY(dalloc(&m.cell_atoms, N));
            CUDA_TRY(dalloc(&m.cell_q, N));
        } else {                           // fixed-capacity cells: twice the mean occupancy plus 16, grown on overflow
            m.ccap = ((int)(2.0 * N / m.n_cells) + 16 + 7) / 8 * 8;
            CUDA_TRY(dalloc(&m.cell_atoms, (size_t)m.n_cells * m.ccap));
            CUDA_TRY(dalloc(&m.cell_q, (size_t)m.n_cells * m.ccap));
        }
    }
    CUDA_TRY(alloc_model_nbr(c, m));
    CUDA_TRY(dalloc(&m.nbr_cnt, N));
    CUDA_TRY(dalloc(&m.vl_cnt, N));
    {   // folded row scan: a pair count per build block of 8 atoms and per chunk of 32 blocks
        const size_t nb = (size_t)(N + 7) / 8, nch = (nb + 31) / 32 + 1;
        CUDA_TRY(dalloc(&m.block_sum, nb));
        CUDA_TRY(dalloc(&m.chunk_sum, nch));
        CUDA_TRY(dalloc(&m.ticket, 1));
        CUDA_TRY(cudaMemset(m.chunk_sum, 0, sizeof(int) * nch));
        CUDA_TRY(cudaMemset(m.ticket, 0, sizeof(unsigned int)));
    }
    CUDA_TRY(dalloc(&m.row_ptr, N + 1));
    size_t nf = (size_t)N * m.F;
    CUDA_TRY(dalloc(&m.h, nf));
    CUDA_TRY(dalloc(&m.h0, nf));
    CUDA_TRY(dalloc(&m.gh, nf));
    for (int l = 0; l < m.L; ++l) {
        CUDA_TRY(dalloc(&m.u[l], nf));
        CUDA_TRY(dalloc(&m.z[l], nf));
        CUDA_TRY(dalloc(&m.um[l], nf * 4));
    }
    CUDA_TRY(dalloc(&m.mbar[0], nf));
    CUDA_TRY(dalloc(&m.mbar[1], nf));
    CUDA_TRY(dalloc(&m.msg, nf));
    CUDA_TRY(dalloc(&m.force, (size_t)3 * N));
    CUDA_TRY(cudaMemset(m.force, 0, sizeof(float) * 3 * std::max(N, 1)));
    CUDA_TRY(dalloc(&m.vir6, (size_t)6 * N));
    CUDA_TRY(dalloc(&m.Ei, N));
    CUDA_TRY(dalloc(&m.erep, N));
    CUDA_TRY(dalloc(&m.E, c->n_sys));
    CUDA_TRY(dalloc(&m.esum.part, (size_t)kSumMaxSplit * kSumChunks));
    CUDA_TRY(dalloc(&m.esum.ctr, kSumMaxSplit));
    CUDA_TRY(cudaMemset(m.esum.ctr, 0, sizeof(unsigned int) * kSumMaxSplit));
    CUDA_TRY(dalloc(&m.W, (size_t)9 * c->n_sys));
    // FP32: atoms per CTA (bounded by shared memory); BF16: atoms per chunk of
    // the persistent kernels
    int mf = max_atoms_per_cta_f32(m.F, m.K, false);
    int mb = max_atoms_per_cta_f32(m.F, m.K, true);
    int want = m.F == 64 ? 16 : 32;
    m.apc_fwd = std::max(8, std::min(want, mf));
    m.apc_bwd = std::max(8, std::min(want, mb));
    return DMTS_OK;
}

NbrArgs nbr_args(dmts_ctx* c, Model& m, int which) {
    NbrArgs a{};
    a.n_atoms = c->N;
    a.n_sys = c->n_sys;
    a.q = c->d_q;
    a.x = c->d_x;
    a.atom_offset = c->d_off;
    a.box = c->d_box;
    a.frame = c->d_frame;
    a.rc = m.rc;
    double rc2 = m.rc * m.rc;
    a.rc2_lo = (float)(rc2 * (1.0 - 1e-5));
    a.rc2_hi = (float)(rc2 * (1.0 + 1e-5));
    a.nc = m.nc;
    a.cell_start = m.cell_start;
    a.cell_atoms = m.cell_atoms;
    a.cell_q = m.cell_q;
    a.atom_pos = m.atom_pos;
    a.row_cap = m.row_cap;
    a.e_cap = m.e_cap;
    a.nbr_tmp = m.nbr_tmp;
    a.nbr_cnt = m.nbr_cnt;
    a.row_ptr = m.row_ptr;
    a.col = m.col;
    a.recv = m.recv;
    a.flags = c->d_flags;
    a.which = which;
    a.exact = 1;
    a.flag_row = kFlagMaxRow0 + which;
    a.ccap = m.ccap;
    a.placed = m.placed ? 1 : 0;
    a.n_cells = m.nc > 0 ? m.n_cells : 0;
    a.cell_count = m.cell_count;
    if (c->skin <= 0) {                    // fresh builds fold the row scan into the compaction
        a.block_sum = m.block_sum;
        a.chunk_sum = m.chunk_sum;
        a.ticket = m.ticket;
    }
    return a;
}

PotArgs pot_args(dmts_ctx* c, Model& m) {
    PotArgs a{};
    a.check = c->d_flags;
    a.energy = 1;
    a.P = m.P;
    a.off = m.off;
    a.n_layers = m.L;
    a.n_atoms = c->N;
    a.q = c->d_q;
    a.frame = c->d_frame;
    a.species = c->d_species;
    a.row_ptr = m.row_ptr;
    a.col = m.col;
    a.recv = m.recv;
    a.e_cap = m.e_cap;
    a.rc = (float)m.rc;
    a.pi_over_rc = (float)(M_PI / m.rc);
    a.bessel_pref = (float)sqrt(2.0 / m.rc);
    a.rep_a = (float)m.rep_a;
    a.rep_inv_rho = (float)(1.0 / m.rep_rho);
    a.rep_rc = (float)m.rep_rc;
    a.rep_pi_over_rc = m.rep_rc > 0 ? (float)(M_PI / m.rep_rc) : 0.f;
    a.erep = m.erep;
    a.msg_out = m.msg;
    a.wt = m.wt;
    a.wt_layer_bytes = m.wt_layer_bytes;
    a.PT = m.PT;
    a.at = m.at;
    a.carry = m.carry;
    a.carry_w = m.F + 16;
    a.h = m.h;
    a.h_in = m.h;
    a.gh = m.gh;
    a.Ei = m.Ei;
    a.force = m.force;
    a.vir6 = m.vir6;
    return a;
}

// Position-independent per-atom inputs of one model: h^0 = A[Z_i] and
// u^0 = h^0 W_in^0. Run after every parameter upload.
int prepare_embedding(dmts_ctx* c, Model& m) {
    if (!m.present || c->N == 0) return DMTS_OK;
    PotArgs a = pot_args(c, m);
    a.h = m.h0;
    a.u_next = m.u[0];
    a.um_u_out = m.um[0];
    launch_embed(a, m.F, c->stream);
    CUDA_TRY(cudaGetLastError());
    return DMTS_OK;
}

// Candidate-row arguments of model w at rc + skin (FP32 bound, no exact test).
NbrArgs candidate_args(dmts_ctx* c, int w) {
    Model& m = c->m[w];
    NbrArgs a = nbr_args(c, m, w);
    const double rv = m.rc + c->skin;
    a.rc = rv;
    a.exact = 0;
    a.rc2_lo = a.rc2_hi = (float)(rv * rv * (1.0 + 1e-5));
    a.row_cap = m.vl_cap;
    a.nbr_tmp = m.vl_rows;
    a.nbr_cnt = m.vl_cnt;
    a.flag_row = kFlagMaxVl0 + w;
    a.gate = &c->d_vl->rebuild;
    a.block_sum = nullptr;
    a.chunk_sum = nullptr;
    a.ticket = nullptr;
    return a;
}

// Thermostat parameters for inner steps of length h (fs).
Langevin langevin(dmts_ctx* c, double h) {
    Langevin lg{};
    lg.step = c->d_rng;
    if (!(c->friction_ps > 0.0)) return lg;
    const double gamma = c->friction_ps * 1e-3;             // 1/fs
    lg.on = 1;
    lg.c1 = exp(-gamma * h);
    lg.c2 = sqrt(1.0 - lg.c1 * lg.c1);
    lg.kT_accel = 8.617333262e-5 * c->temperature * accel_constant();
    lg.key0 = (uint32_t)(c->seed & 0xffffffffull);
    lg.key1 = (uint32_t)(c->seed >> 32);
    return lg;
}

VerletCheck verlet_check(dmts_ctx* c) {
    VerletCheck vc{};
    if (c->skin <= 0) return vc;
    vc.xref = c->d_xref;
    vc.st = c->d_vl;
    vc.thr2 = c->vl_thr2;
    return vc;
}

// The gated rebuild of both models' candidate rows (cells, candidate build
// of the model with the larger cutoff, filter of the other's).
void enqueue_rebuild(dmts_ctx* c, cudaStream_t s) {
    const int w0 = c->vl_src;
    Model& src = c->m[w0];
    NbrArgs b = candidate_args(c, w0);
    if (src.nc > 0)
        launch_cells_gated(c->N, c->d_q, src.nc, src.cell_count, src.cell_start, src.cell_atoms, src.atom_cell,
                           src.atom_slot, src.cell_q, src.atom_pos, b.gate, s);
    b.xref = c->d_xref;
    launch_vl_build(b, s);
    if (c->m[1 - w0].present) {
        NbrArgs d = candidate_args(c, 1 - w0);
        d.src_rows = src.vl_rows;
        d.src_cnt = src.vl_cnt;
        d.src_cap = src.vl_cap;
        launch_row_filter(d, s);
    }
}

enum class Check {
    None,     // positions unchanged since the last check: filter only
    Kernel,   // run the displacement check, then the (gated) rebuild
    Done      // the integrator kernel that moved the atoms has checked
};

// Quantise (optionally) and build the neighbour list of one model.
// Stream-ordered, no host synchronisation. With a skin, a check that trips
// rebuilds both models' candidate rows (the rebuild kernels are always
// enqueued, also inside captured graphs, and return at once when the check
// did not trip); the exact filter of the candidate rows always runs.
// (Measured on 12,288-atom water: a conditional graph node around the
// rebuild costs more than the idle rebuild kernels it would skip.)
void enqueue_neighbors(dmts_ctx* c, int which, bool quantize, Check check = Check::Kernel) {
    Model& m = c->m[which];
    cudaStream_t s = c->stream;
    if (quantize) {
        if (!c->periodic) launch_frames(c->n_sys, c->d_off, c->d_x, c->N, c->d_box, c->rc_max, c->d_frame, s);
        launch_quantize(c->N, c->d_x, c->d_sys, c->d_frame, c->d_q, s);
    }
    if (c->skin <= 0) {
        launch_neighbors(nbr_args(c, m, which), s);     // places the atoms into the cells first
        return;
    }
    if (check == Check::Kernel) launch_vl_check(c->N, c->d_x, c->d_sys, c->d_box, verlet_check(c), s);
    if (check != Check::None) enqueue_rebuild(c, s);
    NbrArgs f = nbr_args(c, m, which);
    f.src_rows = m.vl_rows;
    f.src_cnt = m.vl_cnt;
    f.src_cap = m.vl_cap;
    launch_vl_filter(f, s);
}

int force_rebuild(dmts_ctx* c) {
    if (c->skin <= 0) return DMTS_OK;
    CUDA_TRY(cudaMemsetAsync(&c->d_vl->force, 1, sizeof(int), c->stream));
    return DMTS_OK;
}

void launch_edge_fwd(dmts_ctx* c, Model& m, const PotArgs& a) {
    if (m.precision == DMTS_BF16_MLP) launch_edge_fwd_bf16(a, m.F, m.K, c->d_flags + kFlagTimeout, c->stream);
    else launch_edge_fwd_f32(a, m.F, m.K, c->stream);
}

// Per-atom MLPs: tensor cores in the BF16 precision mode for F >= 64
// (unless the option atom_tensor_cores is 0), FP32 SIMT otherwise. At F = 32
// the SIMT kernels measured faster (16 vs 17 us for 12,288 atoms): the
// tensor-core kernels' fixed cost is not repaid by their half-size products.
bool atom_on_tc(const dmts_ctx* c, const Model& m) {
    return m.precision == DMTS_BF16_MLP && c->atom_tc && m.F >= 64;
}

void launch_atom_fwd_m(dmts_ctx* c, Model& m, const PotArgs& a) {
    if (atom_on_tc(c, m)) launch_atom_fwd_tc(a, m.F, m.msg, c->d_flags + kFlagTimeout, c->stream);
    else launch_atom_fwd(a, m.F, m.msg, c->stream);
}

void launch_atom_bwd_m(dmts_ctx* c, Model& m, const PotArgs& a) {
    if (atom_on_tc(c, m)) launch_atom_bwd_tc(a, m.F, m.msg, c->d_flags + kFlagTimeout, c->stream);
    else launch_atom_bwd(a, m.F, m.msg, c->stream);
}

void launch_edge_bwd(dmts_ctx* c, Model& m, const PotArgs& a) {
    if (m.precision == DMTS_BF16_MLP) launch_edge_bwd_bf16(a, m.F, m.K, c->d_flags + kFlagTimeout, c->stream);
    else launch_edge_bwd_f32(a, m.F, m.K, c->stream);
}

// Arguments of layer l's forward pass (edge kernel, then atom MLP) and
// backward pass (edge kernel, then atom MLP for l > 0).
PotArgs fwd_args(dmts_ctx* c, const PotArgs& a, Model& m, int l) {
    PotArgs f = a;
    f.layer = l;
    f.h_in = l == 0 ? m.h0 : m.h;
    f.atoms_per_cta = m.apc_fwd;
    f.ctas_per_sm = m.cps_fwd;
    f.u = m.u[l];
    f.u_next = (l + 1 < m.L) ? m.u[l + 1] : nullptr;
    f.z = m.z[l];
    f.mbar_out = m.mbar[(m.L - 1) & 1];
    // the SIMT per-atom kernel after a tensor-core forward pass sums the split
    // rows itself (one launch fewer); the tensor-core one reads finished rows
    f.fused_fixup = (m.precision == DMTS_BF16_MLP && !atom_on_tc(c, m) && !c->keep_msg) ? 1 : 0;
    if (m.precision == DMTS_BF16_MLP) {
        f.um_u_out = (l + 1 < m.L) ? m.um[l + 1] : nullptr;
        f.um_mbar_out = m.um[m.L - 1];
    }
    return f;
}

PotArgs bwd_args(const PotArgs& a, Model& m, int l) {
    PotArgs b = a;
    b.layer = l;
    b.atoms_per_cta = m.apc_bwd;
    b.ctas_per_sm = m.cps_bwd;
    b.bwd_tiles = m.bwd_tiles;
    b.u = m.u[l];
    b.mbar = m.mbar[l & 1];
    b.mbar_out = (l > 0) ? m.mbar[(l - 1) & 1] : nullptr;
    b.z_prev = (l > 0) ? m.z[l - 1] : nullptr;
    b.accumulate = (l < m.L - 1) ? 1 : 0;
    b.um = m.um[l];
    if (m.precision == DMTS_BF16_MLP) b.um_mbar_out = (l > 0) ? m.um[l - 1] : nullptr;
    return b;
}

// sum_energy false: the per-atom energies are computed but summed elsewhere
// (the closing kernel's fused energy epilogue).
void enqueue_eval(dmts_ctx* c, int which, bool quantize, bool energy = true, Check check = Check::Kernel,
                  bool virial = false, bool sum_energy = true) {
    Range nvtx_range(which == DMTS_BIG ? "evaluate big model" : "evaluate small model");
    Model& m = c->m[which];
    cudaStream_t s = c->stream;
    enqueue_neighbors(c, which, quantize, check);
    PotArgs a = pot_args(c, m);
    a.virial = virial ? 1 : 0;
    a.energy = energy ? 1 : 0;
    a.lean = (which == DMTS_SMALL && c->fold_small && !energy && !virial) ? 1 : 0;   // inside a captured step
    for (int l = 0; l < m.L; ++l) {
        PotArgs f = fwd_args(c, a, m, l);
        launch_edge_fwd(c, m, f);
        launch_atom_fwd_m(c, m, f);
    }
    for (int l = m.L - 1; l >= 0; --l) {
        PotArgs b = bwd_args(a, m, l);
        // inside a captured step the integrator kernels that read F_small sum
        // its rows split across tiles (no separate fix-up pass)
        b.fold_fixup = (which == DMTS_SMALL && c->fold_small && l == 0 && !b.accumulate && !virial &&
                        m.precision == DMTS_BF16_MLP) ? 1 : 0;
        launch_edge_bwd(c, m, b);
        if (l > 0) launch_atom_bwd_m(c, m, b);
    }
    if (energy && sum_energy) launch_system_sum(c->n_sys, c->d_off, m.Ei, m.E, 1, m.esum, s);
}

int sync_check(dmts_ctx* c) {
    // the flags follow the stream's work into pinned host memory: one wait
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int) * kFlagCount, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->broken = true;
        return fail(DMTS_ERR_CUDA, "CUDA error: %s", cudaGetErrorString(e));
    }
    if (c->h_flags[kFlagCheck]) {            // checked builds only
        c->broken = true;
        return fail(DMTS_ERR_CUDA, "index check failed (source line %d): an index outside its array",
                    c->h_flags[kFlagCheck]);
    }
    if (const int t = c->h_flags[kFlagTimeout]) {
        // bit 0: a bounded wait gave up and its kernel stopped early (results
        // invalid); bit 1: work it had in flight did not finish in time either
        if (t & 2) {
            c->broken = true;
            return fail(DMTS_ERR_TIMEOUT, "a completion wait gave up and in-flight work did not drain");
        }
        c->forces_valid = false;
        CUDA_TRY(cudaMemsetAsync(c->d_flags + kFlagTimeout, 0, sizeof(int), c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        return fail(DMTS_ERR_TIMEOUT, "a bounded completion wait gave up");
    }
    return DMTS_OK;
}

// Grow neighbour capacities from the maxima seen on the device.
int grow_capacity(dmts_ctx* c) {
    for (int w = 0; w < 2; ++w) {
        Model& m = c->m[w];
        if (!m.present) continue;
        int max_row = c->h_flags[kFlagMaxRow0 + w];
        long long max_e = (long long)(unsigned int)c->h_flags[kFlagMaxE0 + w];
        bool grow = false;
        int max_vl = c->h_flags[kFlagMaxVl0 + w];
        if (max_row > m.row_cap) { m.row_cap = std::min(c->N, ((int)(max_row * 1.25) + 63) / 32 * 32); grow = true; }
        if (max_e > m.e_cap) { m.e_cap = (long long)(max_e * 1.25) + 1024; grow = true; }
        if (c->skin > 0 && max_vl > m.vl_cap) { m.vl_cap = std::min(c->N, ((int)(max_vl * 1.25) + 63) / 32 * 32); grow = true; }
        const int max_cell = c->h_flags[kFlagMaxCell0 + w];
        if (m.ccap > 0 && max_cell > m.ccap) {
            m.ccap = ((int)(max_cell * 1.25) + 8 + 7) / 8 * 8;
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            dfree(m.cell_atoms);
            dfree(m.cell_q);
            m.cell_atoms = nullptr;
            m.cell_q = nullptr;
            cudaError_t e = dalloc(&m.cell_atoms, (size_t)m.n_cells * m.ccap);
            if (e == cudaSuccess) e = dalloc(&m.cell_q, (size_t)m.n_cells * m.ccap);
            if (e != cudaSuccess) return fail(DMTS_ERR_OOM, "growing cell capacity: %s", cudaGetErrorString(e));
        }
        if (grow) {
            if (m.row_cap > 6000 || m.vl_cap > 6000)
                return fail(DMTS_ERR_CAPACITY, "neighbour row capacity %d too large", std::max(m.row_cap, m.vl_cap));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            free_model_nbr(m);
            cudaError_t e = alloc_model_nbr(c, m);
            if (e != cudaSuccess) return fail(DMTS_ERR_OOM, "growing neighbour capacity: %s", cudaGetErrorString(e));
        }
    }
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return force_rebuild(c);                // rows reallocated, or truncated by the overflow
}

int reset_flags(dmts_ctx* c) {
    CUDA_TRY(cudaMemsetAsync(c->d_flags, 0, sizeof(int) * kFlagCount, c->stream));
    return DMTS_OK;
}

int copy_in(dmts_ctx* c, double* dst, const double* src, size_t n) {
    cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), k, c->stream));
    return DMTS_OK;
}

int copy_out(dmts_ctx* c, double* dst, const double* src, size_t n) {
    cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), k, c->stream));
    return DMTS_OK;
}

// The single-time-step fallback of one outer step (body of the IF node):
// restore x, v and the large-model force saved at the start of the step, take
// n_inner velocity-Verlet (BAOAB) steps of dt / n_inner with the large model,
// drawing the noise of the inner steps they replace, then evaluate the small
// model at the final positions for the next step's kicks.
void enqueue_fallback(dmts_ctx* c, int n_inner, double dt) {
    const double acc = accel_constant();
    const double h = dt / n_inner;
    const bool nonper = !c->periodic;
    launch_copy_state(c->N, c->d_sx, c->d_sv, c->d_sf, c->d_x, c->d_v, c->m[1].force, c->stream);
    Langevin lg = langevin(c, h);
    for (int k = 0; k < n_inner; ++k) {
        lg.offset = (long long)k - n_inner;              // the counter was advanced by the step's closing kernel
        launch_vv_pre(c->N, 0.5 * h * acc, h, c->d_x, c->d_v, c->d_inv_m, c->m[1].force, c->d_sys, c->d_box,
                      c->d_frame, c->d_q, c->d_flags, verlet_check(c), lg, c->stream);
        enqueue_eval(c, 1, nonper, true, Check::Done);
        launch_vv_post(c->N, 0.5 * h * acc, c->d_v, c->d_inv_m, c->m[1].force, c->d_x, c->d_ke, c->d_mass,
                       c->d_flags, nullptr, EnergyFuse{}, c->stream);
    }
    enqueue_eval(c, 0, false, false, Check::None);
}

// During stream capture: an IF node on `h` whose body is the fallback,
// captured on the auxiliary stream; the capture continues after the node.
cudaError_t capture_fallback_node(dmts_ctx* c, cudaGraphConditionalHandle h, int n_inner, double dt) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(c->stream, &st, nullptr, &g, &deps, &ed, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, ed, nd, &p)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCaptureToGraph(c->aux, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
    const cudaStream_t main = c->stream;
    const long long before = c->launches;
    c->stream = c->aux;                        // every launcher enqueues on c->stream
    enqueue_fallback(c, n_inner, dt);
    c->stream = main;
    c->body_launches = c->launches - before;
    c->launches = before;                      // counted when a body runs
    cudaGraph_t body = nullptr;
    if ((e = cudaStreamEndCapture(c->aux, &body)) != cudaSuccess) return e;
    return cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Cells of model w for the integrator kernel to fill (periodic systems with
// fresh lists, whose fixed-point positions that kernel writes); nc = 0: none.
CellPlace cell_place(dmts_ctx* c, int w) {
    const Model& m = c->m[w];
    CellPlace p{};
    if (c->periodic && c->skin <= 0 && m.present && m.nc > 0 && m.ccap > 0)
        p = CellPlace{m.nc, m.ccap, m.cell_count, m.cell_atoms, m.cell_q, m.atom_pos, kFlagMaxCell0 + w};
    return p;
}

// F_small as the integrator kernels of a captured step read it (ForceFold).
ForceFold small_fold(dmts_ctx* c) {
    const Model& m = c->m[0];
    if (!c->fold_small) return ForceFold{};
    return ForceFold{m.row_ptr, m.e_cap, m.carry, m.F + 16, m.F};
}

int capture_step_graph(dmts_ctx* c, int n_inner, double dt) {
    struct PlacedReset {                       // no evaluation outside this capture skips its placement
        dmts_ctx* c;                           // or its force fix-up
        ~PlacedReset() { c->m[0].placed = c->m[1].placed = false; c->fold_small = false; }
    } placed_reset{c};
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    cudaStream_t s = c->stream;
    const double acc = accel_constant();
    long long before = c->launches;
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const bool nonper = !c->periodic;
    cudaError_t ce = cudaSuccess;
    // the integrator kernels that move the atoms also run the neighbour-list
    // displacement check (with a skin)
    const VerletCheck vc = verlet_check(c);
    // one system, no fallback: the closing kernel sums the energies and writes the record
    const bool fuse_e = c->n_sys == 1 && c->fb_threshold <= 0.0;
    EnergyFuse ef{};
    if (fuse_e)
        ef = EnergyFuse{1, c->m[1].Ei, c->m[1].E, c->d_ekin, c->d_epart, c->d_eticket, c->d_ring, c->ring_len};
    if (c->m[0].present) {
        double h = dt / n_inner;
        Langevin lg = langevin(c, h);
        const bool fallback = c->fb_threshold > 0.0;
        MonitorArgs mon{c->d_mon, c->fb_threshold, 0, 0};
        if (fallback) {
            cudaGraph_t g = nullptr;
            cudaStreamCaptureStatus st;
            ce = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
            if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&mon.cond, g, 0, cudaGraphCondAssignDefault);
            mon.use_cond = 1;
            launch_copy_state(c->N, c->d_x, c->d_v, c->m[1].force, c->d_sx, c->d_sv, c->d_sf, s);
        }
        // with fresh neighbour lists the two evaluations at the final positions
        // share nothing but the read-only positions: fork the large one
        const bool fork = c->concurrent && c->skin <= 0;
        // the small model's cells at every inner step, and the large model's
        // at the last, are filled by the integrator kernel (each placement is
        // followed by that model's build, whose compaction empties the cells)
        const CellPlace none{};
        const CellPlace cp0 = cell_place(c, 0), cp1 = cell_place(c, 1);
        c->fold_small = c->m[0].precision == DMTS_BF16_MLP;
        const ForceFold fold = small_fold(c);
        for (int k = 0; k < n_inner; ++k) {
            lg.offset = k;
            const bool last = k == n_inner - 1;
            launch_respa_pre(c->N, k == 0, 0.5 * dt * acc, 0.5 * h * acc, 0.5 * h, c->d_x, c->d_v, c->d_inv_m,
                             c->m[0].force, c->m[1].force, c->d_sys, c->d_box, c->d_frame, c->d_q, c->d_flags, vc,
                             lg, cp0, last ? cp1 : none, fold, s);
            c->m[0].placed = cp0.nc > 0;
            c->m[1].placed = last && cp1.nc > 0;
            if (fork && k == n_inner - 1) {
                if (nonper) {                                  // frames and fixed-point positions for both
                    launch_frames(c->n_sys, c->d_off, c->d_x, c->N, c->d_box, c->rc_max, c->d_frame, s);
                    launch_quantize(c->N, c->d_x, c->d_sys, c->d_frame, c->d_q, s);
                }
                CUDA_TRY(cudaEventRecord(c->ev_fork, s));
                CUDA_TRY(cudaStreamWaitEvent(c->s_big, c->ev_fork, 0));
                c->stream = c->s_big;                          // every launcher enqueues on c->stream
                enqueue_eval(c, 1, false, true, Check::None, false, !fuse_e);
                c->stream = s;
                CUDA_TRY(cudaEventRecord(c->ev_join, c->s_big));
                enqueue_eval(c, 0, false, false, Check::None);
                CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
            } else {
                enqueue_eval(c, 0, nonper, false, Check::Done);   // the small model's energy is not reported
            }
        }
        if (!fork) enqueue_eval(c, 1, false, true, Check::None, false, !fuse_e);   // same positions as the last small evaluation
        c->m[0].placed = c->m[1].placed = false;
        launch_respa_post(c->N, 0.5 * dt * acc, 0.5 * h * acc, c->d_v, c->d_inv_m, c->m[0].force,
                          c->m[1].force, c->d_x, c->d_ke, c->d_mass, c->d_flags, c->d_rng, n_inner, mon, fold, ef, s);
        c->fold_small = false;                 // the fallback body completes its own forces
        if (fallback && ce == cudaSuccess) ce = capture_fallback_node(c, mon.cond, n_inner, dt);
    } else {
        launch_vv_pre(c->N, 0.5 * dt * acc, dt, c->d_x, c->d_v, c->d_inv_m, c->m[1].force, c->d_sys, c->d_box,
                      c->d_frame, c->d_q, c->d_flags, vc, langevin(c, dt), s);
        enqueue_eval(c, 1, nonper, true, Check::Done, false, !fuse_e);
        launch_vv_post(c->N, 0.5 * dt * acc, c->d_v, c->d_inv_m, c->m[1].force, c->d_x, c->d_ke, c->d_mass,
                       c->d_flags, c->d_rng, ef, s);
    }
    if (!fuse_e) {
        launch_system_sum(c->n_sys, c->d_off, c->d_ke, c->d_ekin, 1, c->kesum, s);
        launch_energy_record(c->n_sys, c->m[1].E, c->d_ekin, c->d_ring, c->ring_len, c->d_flags, s);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = ce;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        c->broken = true;
        return fail(DMTS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->broken = true;
        return fail(DMTS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    c->g_nodes = c->launches - before;
    c->launches = before;
    c->g_n_inner = n_inner;
    c->g_dt = dt;
    return DMTS_OK;
}

// Autotuner: times one force evaluation of each model for a few work
// granularities (atoms per CTA for the FP32 kernels, persistent CTAs per SM
// for the tensor-core kernels) and keeps the fastest forward and backward
// edge pass. The FP32 kernels sum every atom's row in edge order whatever the
// granularity; the tensor-core kernels cut the pair list into the same fixed
// 128-pair tiles whatever the grid and sum split rows in tile order. So the
// results are bit-identical for every candidate. Runs once per context, at
// the first evaluation.
int time_stages_impl(dmts_ctx* c, int which, int reps, std::vector<double>& acc);

int autotune_models(dmts_ctx* c) {
    if (!c->autotune || c->tuned) return DMTS_OK;
    int rc = DMTS_OK;
    for (int w = 0; w < 2 && rc == DMTS_OK; ++w) {
        Model& m = c->m[w];
        if (!m.present) continue;
        const bool tc = m.precision == DMTS_BF16_MLP;
        // tensor-core kernels: persistent CTAs per SM, and the backward
        // kernel's tiles in flight per CTA (one, or two sharing the weights);
        // FP32 kernels: atoms per CTA
        std::vector<int> tiles_c = tc ? std::vector<int>{1, 2} : std::vector<int>{0};
        int& gf = tc ? m.cps_fwd : m.apc_fwd;
        int& gb = tc ? m.cps_bwd : m.apc_bwd;
        double best_tf = 1e30, best_tb = 1e30;
        int best_f = gf, best_b = gb, best_t = m.bwd_tiles;
        for (int tiles : tiles_c) {
            const int lim_f = tc ? bf16_max_ctas_per_sm(m.F, false) : max_atoms_per_cta_f32(m.F, m.K, false);
            const int lim_b = tc ? bf16_max_ctas_per_sm(m.F, true, tiles) : max_atoms_per_cta_f32(m.F, m.K, true);
            std::vector<int> cand;
            if (tc) for (int k = 1; k <= std::max(lim_f, lim_b); ++k) cand.push_back(k);
            else cand = m.F == 64 ? std::vector<int>{8, 16, 24} : std::vector<int>{16, 32, 48};
            m.bwd_tiles = tiles;
            for (int A : cand) {
                gf = std::min(A, lim_f);
                gb = std::min(A, lim_b);
                std::vector<double> st;
                if ((rc = time_stages_impl(c, w, 3, st))) break;   // sizes capacities, then times the stages
                double tf = 0.0, tb = 0.0;                          // forward and backward edge passes
                for (int l = 0; l < m.L; ++l) {
                    tf += st[2 + l];
                    tb += st[2 + 2 * m.L + l];
                }
                if (tf < best_tf) { best_tf = tf; best_f = gf; }
                if (tb < best_tb) { best_tb = tb; best_b = gb; best_t = tiles; }
            }
            if (rc) break;
        }
        gf = best_f;
        gb = best_b;
        m.bwd_tiles = best_t;
    }
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    c->tuned = true;
    return rc;
}

#define CTX_GUARD(c)                                                                         \
    do {                                                                                     \
        if (!(c)) return fail(DMTS_ERR_ARG, "context is NULL");                              \
        if ((c)->broken) return fail(DMTS_ERR_STATE, "context is unusable after a CUDA error"); \
        cudaSetDevice((c)->device);                                                          \
    } while (0)

}  // namespace

namespace dmts {
void set_error_message(const char* msg) { g_err = msg ? msg : ""; }

ModelOffsets model_offsets(int S, int F, int K, int L) {
    ModelOffsets o{};
    int p = 0;
    o.A = p; p += S * F;
    for (int l = 0; l < L; ++l) {
        o.W_in[l] = p; p += F * F;
        o.W1[l] = p; p += K * F;
        o.b1[l] = p; p += F;
        o.W2[l] = p; p += F * F;
        o.b2[l] = p; p += F;
        o.U1[l] = p; p += F * F;
        o.c1[l] = p; p += F;
        o.U2[l] = p; p += F * F;
        o.c2[l] = p; p += F;
    }
    o.R1 = p; p += F * F;
    o.d1 = p; p += F;
    o.R2 = p; p += F;
    o.d2 = p; p += 1;
    o.e0 = p; p += S;
    o.total = p;
    return o;
}
}  // namespace dmts

extern "C" {

const char* dmts_last_error(void) { return g_err.c_str(); }

void dmts_destroy(dmts_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    free_model(c->m[0]);
    free_model(c->m[1]);
    dfree(c->d_off); dfree(c->d_species); dfree(c->d_sys); dfree(c->d_box); dfree(c->d_mass);
    dfree(c->d_inv_m); dfree(c->d_x); dfree(c->d_v); dfree(c->d_q); dfree(c->d_frame); dfree(c->d_stage);
    dfree(c->d_ke); dfree(c->d_ekin); dfree(c->d_ring); dfree(c->d_flags); dfree(c->d_epart); dfree(c->d_eticket);
    dfree(c->d_bx); dfree(c->d_bv);
    dfree(c->d_xref); dfree(c->d_vl); dfree(c->d_rng); dfree(c->kesum.part); dfree(c->kesum.ctr);
    dfree(c->d_mon); dfree(c->d_sx); dfree(c->d_sv); dfree(c->d_sf);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->s_big) cudaStreamDestroy(c->s_big);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    dfree(c->fm_g); dfree(c->fm_m); dfree(c->fm_mdot); dfree(c->fm_mb); dfree(c->fm_mdb); dfree(c->fm_ubar);
    dfree(c->fm_pe); dfree(c->fm_pa); dfree(c->fm_sq); dfree(c->fm_grad); dfree(c->fm_loss); dfree(c->fm_stage);
    dfree(c->fm_eref); dfree(c->fm_ce);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int dmts_create(const dmts_model_desc* small, const dmts_model_desc* big, const dmts_system_desc* sys,
                const char* options, dmts_ctx** out) {
    Range nvtx_range("dmts_create");
    g_err.clear();
    if (!out) return fail(DMTS_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_model(big, "big");
    if (rc) return rc;
    if (small && (rc = check_model(small, "small"))) return rc;
    if (!sys || sys->n_systems < 1 || !sys->atom_offset || !sys->species || !sys->mass || !sys->box)
        return fail(DMTS_ERR_ARG, "system descriptor incomplete");
    const int ns = sys->n_systems;
    if (sys->atom_offset[0] != 0) return fail(DMTS_ERR_ARG, "atom_offset[0] must be 0");
    for (int s = 0; s < ns; ++s)
        if (sys->atom_offset[s + 1] < sys->atom_offset[s]) return fail(DMTS_ERR_ARG, "atom_offset must be non-decreasing");
    const int N = sys->atom_offset[ns];
    double rc_max = std::max(big->cutoff, small ? small->cutoff : 0.0);
    int n_per = 0;
    for (int s = 0; s < ns; ++s) {
        double L = sys->box[s];
        if (!isfinite(L)) return fail(DMTS_ERR_ARG, "box[%d] not finite", s);
        if (L > 0) {
            ++n_per;
            if (L < 2.0 * rc_max) return fail(DMTS_ERR_ARG, "box edge %g is below twice the cutoff %g", L, rc_max);
        } else if (sys->atom_offset[s + 1] - sys->atom_offset[s] > kMaxMolAtoms) {
            return fail(DMTS_ERR_ARG, "non-periodic system %d has more than %d atoms", s, kMaxMolAtoms);
        }
    }
    if (n_per > 0 && n_per != ns) return fail(DMTS_ERR_ARG, "periodic and non-periodic systems cannot be mixed");
    for (int s = 1; s < n_per; ++s)
        if (sys->box[s] != sys->box[0]) return fail(DMTS_ERR_ARG, "periodic systems must share one box edge");
    int S_min = std::min(big->n_species, small ? small->n_species : 1 << 30);
    for (int i = 0; i < N; ++i) {
        if (sys->species[i] < 0 || sys->species[i] >= S_min) return fail(DMTS_ERR_ARG, "species[%d] out of range", i);
        if (!(sys->mass[i] > 0) || !isfinite(sys->mass[i])) return fail(DMTS_ERR_ARG, "mass[%d] must be > 0", i);
    }
    Options opt;
    if ((rc = parse_options(options, opt))) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(DMTS_ERR_CUDA, "no CUDA device available");
    }
    dmts_ctx* c = new dmts_ctx();
    cudaGetDevice(&c->device);
    LaunchScope ls(c);
    c->N = N;
    c->n_sys = ns;
    c->periodic = n_per > 0;
    c->h_off.assign(sys->atom_offset, sys->atom_offset + ns + 1);
    c->h_box.assign(sys->box, sys->box + ns);
    c->rc_max = rc_max;
    c->autotune = opt.get("autotune", 1.0) != 0.0;
    c->cap_factor = opt.get("edge_capacity_factor", 1.5);
    if (!(c->cap_factor > 0.0)) c->cap_factor = 1.5;
    const double opt_row_cap = opt.get("row_capacity", 0.0);
    const double opt_cell_cap = opt.get("cell_capacity", 0.0);
    c->skin = opt.get("skin", 0.0);
    if (!(c->skin >= 0.0) || c->skin > 10.0) {
        delete c;
        return fail(DMTS_ERR_ARG, "skin must be in [0, 10] A");
    }
    c->vl_thr2 = 0.25 * c->skin * c->skin * (1.0 - 2e-3);
    c->friction_ps = opt.get("langevin_friction", 0.0);
    c->temperature = opt.get("temperature", 300.0);
    const double seed_d = opt.get("seed", 0.0);
    if (!(c->friction_ps >= 0.0) || !(c->temperature >= 0.0) || !(seed_d >= 0.0) || seed_d > 9.0e15 ||
        !isfinite(c->friction_ps) || !isfinite(c->temperature)) {
        delete c;
        return fail(DMTS_ERR_ARG, "langevin_friction and temperature must be >= 0, seed in [0, 9e15]");
    }
    c->seed = (unsigned long long)seed_d;
    c->fb_threshold = opt.get("fallback_threshold", 0.0);
    if (!(c->fb_threshold >= 0.0)) {
        delete c;
        return fail(DMTS_ERR_ARG, "fallback_threshold must be >= 0 (eV/A)");
    }
    c->vl_src = (small && small->cutoff > big->cutoff) ? 0 : 1;
#define CREATE_TRY(expr)                                                          \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            int code_ = e_ == cudaErrorMemoryAllocation ? DMTS_ERR_OOM : DMTS_ERR_CUDA; \
            fail(code_, "%s: %s", #expr, cudaGetErrorString(e_));                 \
            std::string keep_ = g_err;                                            \
            dmts_destroy(c);                                                      \
            g_err = keep_;                                                        \
            return code_;                                                         \
        }                                                                         \
    } while (0)
    CREATE_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    std::vector<int> sys_of(N);
    for (int s = 0; s < ns; ++s)
        for (int i = sys->atom_offset[s]; i < sys->atom_offset[s + 1]; ++i) sys_of[i] = s;
    std::vector<double> inv_m(N);
    for (int i = 0; i < N; ++i) inv_m[i] = 1.0 / sys->mass[i];
    CREATE_TRY(dalloc(&c->d_off, ns + 1));
    CREATE_TRY(dalloc(&c->d_species, N));
    CREATE_TRY(dalloc(&c->d_sys, N));
    CREATE_TRY(dalloc(&c->d_box, ns));
    CREATE_TRY(dalloc(&c->d_mass, N));
    CREATE_TRY(dalloc(&c->d_inv_m, N));
    CREATE_TRY(dalloc(&c->d_x, (size_t)3 * N));
    CREATE_TRY(dalloc(&c->d_v, (size_t)3 * N));
    CREATE_TRY(dalloc(&c->d_q, N));
    CREATE_TRY(dalloc(&c->d_frame, ns));
    CREATE_TRY(dalloc(&c->d_stage, (size_t)6 * N));
    CREATE_TRY(dalloc(&c->d_ke, N));
    CREATE_TRY(dalloc(&c->d_ekin, ns));
    CREATE_TRY(dalloc(&c->d_epart, (size_t)2 * std::max(1, integrator_blocks(N))));
    CREATE_TRY(dalloc(&c->d_eticket, 1));
    CREATE_TRY(cudaMemset(c->d_eticket, 0, sizeof(unsigned int)));
    CREATE_TRY(dalloc(&c->d_flags, kFlagCount));
    CREATE_TRY(dalloc(&c->d_bx, (size_t)3 * N));
    CREATE_TRY(dalloc(&c->d_bv, (size_t)3 * N));
    CREATE_TRY(cudaMallocHost((void**)&c->h_flags, sizeof(int) * kFlagCount));
    CREATE_TRY(dalloc(&c->kesum.part, (size_t)kSumMaxSplit * kSumChunks));
    CREATE_TRY(dalloc(&c->kesum.ctr, kSumMaxSplit));
    CREATE_TRY(cudaMemset(c->kesum.ctr, 0, sizeof(unsigned int) * kSumMaxSplit));
    CREATE_TRY(dalloc(&c->d_rng, 2));
    CREATE_TRY(cudaMemset(c->d_rng, 0, 2 * sizeof(unsigned long long)));
    CREATE_TRY(cudaStreamCreateWithFlags(&c->s_big, cudaStreamNonBlocking));
    CREATE_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CREATE_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    c->concurrent = opt.get("concurrent_models", 1.0) != 0.0;
    c->atom_tc = opt.get("atom_tensor_cores", 1.0) != 0.0;
    CREATE_TRY(dalloc(&c->d_mon, 1));
    CREATE_TRY(cudaMemset(c->d_mon, 0, sizeof(ForceMonitor)));
    if (c->fb_threshold > 0.0) {
        CREATE_TRY(dalloc(&c->d_sx, (size_t)3 * N));
        CREATE_TRY(dalloc(&c->d_sv, (size_t)3 * N));
        CREATE_TRY(dalloc(&c->d_sf, (size_t)3 * N));
        CREATE_TRY(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    }
    if (c->skin > 0) {
        CREATE_TRY(dalloc(&c->d_xref, (size_t)3 * N));
        CREATE_TRY(dalloc(&c->d_vl, 1));
        CREATE_TRY(cudaMemset(c->d_vl, 0, sizeof(VerletState)));
        CREATE_TRY(cudaMemset(&c->d_vl->force, 1, sizeof(int)));
    }
    CREATE_TRY(cudaMemcpy(c->d_off, sys->atom_offset, sizeof(int) * (ns + 1), cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(c->d_species, sys->species, sizeof(int) * std::max(N, 0), cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(c->d_sys, sys_of.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(c->d_box, sys->box, sizeof(double) * ns, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(c->d_mass, sys->mass, sizeof(double) * N, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(c->d_inv_m, inv_m.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemset(c->d_x, 0, sizeof(double) * 3 * std::max(N, 1)));
    CREATE_TRY(cudaMemset(c->d_v, 0, sizeof(double) * 3 * std::max(N, 1)));
    CREATE_TRY(cudaMemset(c->d_flags, 0, sizeof(int) * kFlagCount));
    if (small) {
        rc = init_model(c, c->m[0], small, c->skin <= 0 || c->vl_src == 0);
        if (rc) { std::string k = g_err; dmts_destroy(c); g_err = k; return rc; }
        c->m[0].apc_fwd = std::min(c->m[0].apc_fwd, (int)opt.get("atoms_per_cta_small", c->m[0].apc_fwd));
        c->m[0].apc_bwd = std::min(c->m[0].apc_bwd, (int)opt.get("atoms_per_cta_small", c->m[0].apc_bwd));
    }
    rc = init_model(c, c->m[1], big, c->skin <= 0 || c->vl_src == 1);
    if (rc) { std::string k = g_err; dmts_destroy(c); g_err = k; return rc; }
    c->m[1].apc_fwd = std::min(c->m[1].apc_fwd, (int)opt.get("atoms_per_cta_big", c->m[1].apc_fwd));
    c->m[1].apc_bwd = std::min(c->m[1].apc_bwd, (int)opt.get("atoms_per_cta_big", c->m[1].apc_bwd));
    for (int w = 0; w < 2; ++w) {
        if (c->m[w].present && opt_row_cap >= 1.0) {
            // smaller initial row capacity (exercises the overflow-and-retry path)
            c->m[w].row_cap = std::min(c->m[w].row_cap, (int)opt_row_cap);
            c->m[w].vl_cap = std::min(c->m[w].vl_cap, (int)opt_row_cap);
            free_model_nbr(c->m[w]);
            CREATE_TRY(alloc_model_nbr(c, c->m[w]));
        }
        if (c->m[w].present && c->m[w].ccap > 0 && opt_cell_cap >= 1.0) {
            // smaller initial cell capacity (exercises the overflow-and-retry path)
            Model& m = c->m[w];
            m.ccap = std::min(m.ccap, (int)opt_cell_cap);
            dfree(m.cell_atoms);
            dfree(m.cell_q);
            m.cell_atoms = nullptr;
            m.cell_q = nullptr;
            CREATE_TRY(dalloc(&m.cell_atoms, (size_t)m.n_cells * m.ccap));
            CREATE_TRY(dalloc(&m.cell_q, (size_t)m.n_cells * m.ccap));
        }
        c->m[w].apc_fwd = std::max(8, c->m[w].apc_fwd);
        c->m[w].apc_bwd = std::max(8, c->m[w].apc_bwd);
    }
    for (int w = 0; w < 2; ++w) {
        if ((rc = prepare_embedding(c, c->m[w]))) { std::string k = g_err; dmts_destroy(c); g_err = k; return rc; }
    }
    if (c->periodic) {
        // constant frame; computed once on the device
        launch_frames(ns, c->d_off, c->d_x, N, c->d_box, rc_max, c->d_frame, c->stream);
        CREATE_TRY(cudaStreamSynchronize(c->stream));
    }
    CREATE_TRY(cudaGetLastError());
    *out = c;
    return DMTS_OK;
}

int dmts_set_state(dmts_ctx* c, const double* x, const double* v, int n_atoms) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_set_state");
    if (!x) return fail(DMTS_ERR_ARG, "x is NULL");
    if (n_atoms != c->N) return fail(DMTS_ERR_ARG, "n_atoms %d != %d", n_atoms, c->N);
    LaunchScope ls(c);
    size_t n3 = (size_t)3 * c->N;
    int rc = copy_in(c, c->d_stage, x, n3);
    if (rc) return rc;
    if (v && (rc = copy_in(c, c->d_stage + n3, v, n3))) return rc;
    CUDA_TRY(cudaMemsetAsync(c->d_flags + kFlagMoved, 0, sizeof(int), c->stream));
    launch_set_state(c->N, c->d_stage, v ? c->d_stage + n3 : nullptr, c->d_sys, c->d_box, c->d_x, c->d_v,
                     c->d_flags + kFlagMoved, c->stream);
    CUDA_TRY(cudaMemsetAsync(c->d_rng, 0, sizeof(unsigned long long), c->stream));   // noise restarts at step 0
    if ((rc = sync_check(c))) return rc;
    // The forces depend on the positions only, and every evaluation of them is
    // deterministic: forces cached at bit-identical positions stay valid, and
    // only a change of position makes the next step Algorithm 1's first step.
    c->forces_valid = c->forces_valid && c->state_set && c->h_flags[kFlagMoved] == 0;
    c->state_set = true;
    return DMTS_OK;
}

int dmts_get_state(dmts_ctx* c, double* x, double* v) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_get_state");
    LaunchScope ls(c);
    size_t n3 = (size_t)3 * c->N;
    launch_get_state(c->N, c->d_x, c->d_v, c->d_stage, c->d_stage + n3, c->stream);
    int rc;
    if (x && (rc = copy_out(c, x, c->d_stage, n3))) return rc;
    if (v && (rc = copy_out(c, v, c->d_stage + n3, n3))) return rc;
    return sync_check(c);
}

int dmts_forces(dmts_ctx* c, int which, double* f_out, double* energy_out, double* virial_out) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_forces");
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    if (!c->m[which].present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (!c->state_set) return fail(DMTS_ERR_STATE, "no state set");
    LaunchScope ls(c);
    Model& m = c->m[which];
    int rc;
    if ((rc = autotune_models(c))) return rc;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((rc = reset_flags(c))) return rc;
        enqueue_eval(c, which, true, true, Check::Kernel, virial_out != nullptr);
        if (virial_out) launch_virial_sum(c->n_sys, c->d_off, m.vir6, m.W, c->stream);
        if ((rc = sync_check(c))) return rc;
        if (!c->h_flags[kFlagOverflow]) break;
        if ((rc = grow_capacity(c))) return rc;
        if (attempt == 3) return fail(DMTS_ERR_CAPACITY, "neighbour capacity overflow persists");
    }
    size_t n3 = (size_t)3 * c->N;
    if (f_out) {
        launch_forces_out(c->N, m.force, c->d_stage, c->stream);
        if ((rc = copy_out(c, f_out, c->d_stage, n3))) return rc;
    }
    if (energy_out && (rc = copy_out(c, energy_out, m.E, c->n_sys))) return rc;
    if (virial_out && (rc = copy_out(c, virial_out, m.W, (size_t)9 * c->n_sys))) return rc;
    return sync_check(c);
}

int dmts_neighbors(dmts_ctx* c, int which, int* row_ptr, int* col, long long capacity, long long* n_pairs) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_neighbors");
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    if (!c->m[which].present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (!c->state_set) return fail(DMTS_ERR_STATE, "no state set");
    if (!row_ptr || !n_pairs || (capacity > 0 && !col)) return fail(DMTS_ERR_ARG, "NULL output");
    LaunchScope ls(c);
    Model& m = c->m[which];
    int rc;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((rc = reset_flags(c))) return rc;
        enqueue_neighbors(c, which, true);
        if ((rc = sync_check(c))) return rc;
        if (!c->h_flags[kFlagOverflow]) break;
        if ((rc = grow_capacity(c))) return rc;
        if (attempt == 3) return fail(DMTS_ERR_CAPACITY, "neighbour capacity overflow persists");
    }
    int total = 0;
    CUDA_TRY(cudaMemcpy(&total, m.row_ptr + c->N, sizeof(int), cudaMemcpyDeviceToHost));
    *n_pairs = total;
    cudaMemcpyKind k1 = is_device_ptr(row_ptr) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CUDA_TRY(cudaMemcpy(row_ptr, m.row_ptr, sizeof(int) * (c->N + 1), k1));
    if (total > capacity) return fail(DMTS_ERR_CAPACITY, "%d pairs exceed capacity %lld", total, capacity);
    if (total > 0) {
        cudaMemcpyKind k2 = is_device_ptr(col) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CUDA_TRY(cudaMemcpy(col, m.col, sizeof(int) * total, k2));
    }
    return DMTS_OK;
}

int dmts_set_params(dmts_ctx* c, int which, const double* params, size_t n_params) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_set_params");
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    Model& m = c->m[which];
    if (!m.present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (!params || n_params != m.n_params) return fail(DMTS_ERR_ARG, "expected %zu parameters", m.n_params);
    for (size_t k = 0; k < n_params; ++k)
        if (!isfinite(params[k])) return fail(DMTS_ERR_ARG, "parameter %zu is not finite", k);
    int rc = upload_params(c, m, params);
    if (rc) return rc;
    if ((rc = prepare_embedding(c, m))) return rc;
    c->forces_valid = false;
    return DMTS_OK;
}

int dmts_respa_step(dmts_ctx* c, int n_outer, double dt, int n_inner, double* energies_out) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_respa_step");
    if (!c->state_set) return fail(DMTS_ERR_STATE, "no state set");
    if (n_outer < 0) return fail(DMTS_ERR_ARG, "n_outer must be >= 0");
    if (!(dt > 0) || !isfinite(dt)) return fail(DMTS_ERR_ARG, "dt must be > 0");
    if (n_inner < 1 || n_inner > 64) return fail(DMTS_ERR_ARG, "n_inner must be in [1, 64]");
    if (!c->m[0].present && n_inner != 1) return fail(DMTS_ERR_ARG, "without a small model n_inner must be 1");
    if (n_outer == 0) return DMTS_OK;
    LaunchScope ls(c);
    int rc;
    size_t n3 = (size_t)3 * c->N;
    if ((rc = autotune_models(c))) return rc;
    if (n_outer > c->ring_len) {
        dfree(c->d_ring);
        c->d_ring = nullptr;
        c->ring_len = 0;
        if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
        cudaError_t e = dalloc(&c->d_ring, (size_t)n_outer * c->n_sys * 3);
        if (e != cudaSuccess) return fail(DMTS_ERR_OOM, "energies ring: %s", cudaGetErrorString(e));
        c->ring_len = n_outer;
    }
    // state at entry, for the retry after a capacity overflow (the cached
    // forces are not saved: the retry evaluates them again at the restored
    // positions, which gives the same bits, as every evaluation is deterministic)
    CUDA_TRY(cudaMemcpyAsync(c->d_bx, c->d_x, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->d_bv, c->d_v, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->d_rng + 1, c->d_rng, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                             c->stream));
    // back to the state of the call's entry (after an overflow, or a bounded
    // wait that gave up)
    auto restore = [&]() -> int {
        CUDA_TRY(cudaMemcpyAsync(c->d_x, c->d_bx, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->d_v, c->d_bv, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->d_rng, c->d_rng + 1, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                 c->stream));
        c->forces_valid = false;
        return DMTS_OK;
    };
    for (int attempt = 0;; ++attempt) {
        if ((rc = reset_flags(c))) return rc;
        if (!c->forces_valid) {
            // Algorithm 1, first_step: both forces at the current positions
            if (c->m[0].present) enqueue_eval(c, 0, true, false);
            enqueue_eval(c, 1, true);
        }
        if (!c->graph || c->g_n_inner != n_inner || c->g_dt != dt) {
            if ((rc = capture_step_graph(c, n_inner, dt))) return rc;
        }
        for (int s = 0; s < n_outer; ++s) {
            CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
            c->launches += c->g_nodes;
        }
        // this attempt's energies travel with its flags (one wait)
        if (energies_out && (rc = copy_out(c, energies_out, c->d_ring, (size_t)n_outer * c->n_sys * 3))) return rc;
        if ((rc = sync_check(c))) {
            if (rc == DMTS_ERR_TIMEOUT && !c->broken && restore() == DMTS_OK) {
                c->forces_valid = false;
                (void)cudaStreamSynchronize(c->stream);
                set_error_message("a bounded completion wait gave up; the state of the call's entry is restored");
            }
            return rc;
        }
        if (c->fb_threshold > 0.0 && c->m[0].present) {
            // kernels of the fallback bodies that ran
            unsigned long long nf = 0;
            CUDA_TRY(cudaMemcpy(&nf, &c->d_mon->n_fallback, sizeof(nf), cudaMemcpyDeviceToHost));
            c->launches += ((long long)nf - c->fallback_seen) * c->body_launches;
            c->fallback_seen = (long long)nf;
        }
        if (!c->h_flags[kFlagOverflow]) break;
        if (attempt >= 3) return fail(DMTS_ERR_CAPACITY, "neighbour capacity overflow persists");
        // restore and retry with grown capacity
        if ((rc = restore())) return rc;
        if ((rc = grow_capacity(c))) return rc;
    }
    c->forces_valid = true;
    if (c->h_flags[kFlagNonfinite]) return fail(DMTS_ERR_NONFINITE, "non-finite position or velocity");
    return DMTS_OK;
}

void* dmts_stream(dmts_ctx* c) { return c ? (void*)c->stream : nullptr; }

}  // extern "C"

namespace {

// Distillation loss of the small model over n_frames frames and its
// parameter gradient (e_ref null: force matching alone). Every frame is
// enqueued without a host synchronisation; a neighbour overflow in any frame
// grows the capacities and redoes the whole batch.
int distill_impl(dmts_ctx* c, int n_frames, const double* frames, const double* f_ref, const double* e_ref,
                 double lambda_e, double* loss_out, double* grad_out) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_distill_grad");
    Model& m = c->m[0];
    if (!m.present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (!fm_supported(m.F, m.K, m.L))
        return fail(DMTS_ERR_ARG, "distillation needs a single-layer small model with n_feat 32, n_radial 8 or 16");
    if (n_frames < 1 || !frames || !f_ref || !loss_out || !grad_out) return fail(DMTS_ERR_ARG, "bad arguments");
    if (e_ref && !(lambda_e >= 0.0 && isfinite(lambda_e))) return fail(DMTS_ERR_ARG, "lambda_e must be >= 0");
    LaunchScope ls(c);
    const int N = c->N;
    const size_t n3 = (size_t)3 * N, nf = (size_t)N * m.F;
    const int np = (int)m.n_params;
    if (!c->fm_g) {
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = dalloc(&c->fm_g, n3);
        if (e == cudaSuccess) e = dalloc(&c->fm_m, nf);
        if (e == cudaSuccess) e = dalloc(&c->fm_mdot, nf);
        if (e == cudaSuccess) e = dalloc(&c->fm_mb, nf);
        if (e == cudaSuccess) e = dalloc(&c->fm_mdb, nf);
        if (e == cudaSuccess) e = dalloc(&c->fm_ubar, nf);
        if (e == cudaSuccess) e = dalloc(&c->fm_pe, (size_t)fm_edge_ctas(N) * np);
        if (e == cudaSuccess) e = dalloc(&c->fm_pa, (size_t)fm_atom_rows(N) * np);
        if (e == cudaSuccess) e = dalloc(&c->fm_sq, N);
        if (e == cudaSuccess) e = dalloc(&c->fm_grad, np);
        if (e == cudaSuccess) e = dalloc(&c->fm_loss, 1);
        if (e == cudaSuccess) e = dalloc(&c->fm_ce, 1);
        if (e == cudaSuccess) e = dalloc(&c->fm_stage, 2 * n3);
        if (e != cudaSuccess) return fail(DMTS_ERR_OOM, "distillation buffers: %s", cudaGetErrorString(e));
    }
    if (e_ref && n_frames > c->fm_eref_cap) {
        dfree(c->fm_eref);
        c->fm_eref = nullptr;
        c->fm_eref_cap = 0;
        CUDA_TRY(dalloc(&c->fm_eref, (size_t)n_frames));
        c->fm_eref_cap = n_frames;
    }
    int rc;
    if (e_ref && (rc = copy_in(c, c->fm_eref, e_ref, (size_t)n_frames))) return rc;
    // keep the dynamical state
    CUDA_TRY(cudaMemcpyAsync(c->d_bx, c->d_x, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->d_bv, c->d_v, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    // each frame's force and energy come from the model in its own precision
    // (BF16 MLP operands on the tensor cores in DMTS_BF16_MLP mode); the
    // second-order adjoint passes around them are FP32 and read every
    // message row, so the split rows are written back (no fused fix-up)
    struct KeepMsg {
        dmts_ctx* c;
        ~KeepMsg() { c->keep_msg = false; }
    } keep_msg{c};
    c->keep_msg = true;
    const double cl = 2.0 / (3.0 * (double)N * (double)n_frames);
    for (int attempt = 0;; ++attempt) {
        if ((rc = reset_flags(c))) return rc;
        CUDA_TRY(cudaMemsetAsync(c->fm_grad, 0, sizeof(double) * np, c->stream));
        CUDA_TRY(cudaMemsetAsync(c->fm_loss, 0, sizeof(double), c->stream));
        for (int fr = 0; fr < n_frames && N > 0; ++fr) {
            if ((rc = copy_in(c, c->fm_stage, frames + (size_t)fr * n3, n3))) return rc;
            if ((rc = copy_in(c, c->fm_stage + n3, f_ref + (size_t)fr * n3, n3))) return rc;
            // frame positions into x (velocities, saved above, are zeroed meanwhile)
            launch_set_state(N, c->fm_stage, nullptr, c->d_sys, c->d_box, c->d_x, c->d_v, nullptr, c->stream);
            enqueue_eval(c, 0, true, e_ref != nullptr);
            CUDA_TRY(cudaMemcpyAsync(c->fm_m, m.msg, nf * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
            PotArgs a = pot_args(c, m);
            a.layer = 0;
            a.u = m.u[0];                      // u^0 = h0 W_in (gathered per edge)
            if (!a.u || !a.h || !a.force || !a.P || !a.row_ptr || !a.col || !a.recv || !a.q)
                return fail(DMTS_ERR_STATE, "distillation: buffers missing");
            FmEnergy en;
            if (e_ref) {
                en.e_ref = c->fm_eref + fr;
                en.E = m.E;
                en.n_sys = c->n_sys;
                en.lambda = lambda_e;
                en.inv_frames = 1.0 / n_frames;
                en.c_energy = c->fm_ce;
            }
            launch_fm_frame(a, m.K, c->fm_stage + n3, cl, c->fm_g, c->fm_sq, c->fm_m, c->fm_mdot, c->fm_mb,
                            c->fm_mdb, c->fm_ubar, c->fm_pe, c->fm_pa, np, c->fm_grad, c->fm_loss, en,
                            m.precision == DMTS_BF16_MLP, c->d_flags + kFlagTimeout, c->stream);
        }
        if ((rc = sync_check(c))) return rc;
        if (!c->h_flags[kFlagOverflow]) break;
        if (attempt == 3) return fail(DMTS_ERR_CAPACITY, "neighbour capacity overflow persists");
        if ((rc = grow_capacity(c))) return rc;
    }
    CUDA_TRY(cudaMemcpyAsync(c->d_x, c->d_bx, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->d_v, c->d_bv, n3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    c->forces_valid = false;
    if ((rc = copy_out(c, grad_out, c->fm_grad, np))) return rc;
    if ((rc = copy_out(c, loss_out, c->fm_loss, 1))) return rc;
    return sync_check(c);
}

}  // namespace

extern "C" {

int dmts_force_matching_grad(dmts_ctx* c, int n_frames, const double* frames, const double* f_ref,
                             double* loss_out, double* grad_out) {
    return distill_impl(c, n_frames, frames, f_ref, nullptr, 0.0, loss_out, grad_out);
}

int dmts_distill_grad(dmts_ctx* c, int n_frames, const double* frames, const double* f_ref, const double* e_ref,
                      double lambda_e, double* loss_out, double* grad_out) {
    if (!e_ref) return fail(DMTS_ERR_ARG, "e_ref is NULL");
    return distill_impl(c, n_frames, frames, f_ref, e_ref, lambda_e, loss_out, grad_out);
}

int dmts_get_params(dmts_ctx* c, int which, double* params_out, size_t n_params) {
    CTX_GUARD(c);
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    const Model& m = c->m[which];
    if (!m.present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (!params_out || n_params != m.n_params) return fail(DMTS_ERR_ARG, "expected %zu parameters", m.n_params);
    if (is_device_ptr(params_out)) {
        CUDA_TRY(cudaMemcpy(params_out, m.hp.data(), sizeof(double) * n_params, cudaMemcpyHostToDevice));
    } else {
        std::copy(m.hp.begin(), m.hp.end(), params_out);
    }
    return DMTS_OK;
}

int dmts_adam_step(dmts_ctx* c, int which, const double* grad, double* m1, double* m2, long long t, double lr,
                   double beta1, double beta2, double eps) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_adam_step");
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    Model& m = c->m[which];
    if (!m.present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (!grad || !m1 || !m2) return fail(DMTS_ERR_ARG, "NULL argument");
    if (is_device_ptr(m1) || is_device_ptr(m2)) return fail(DMTS_ERR_ARG, "the moment estimates must be host arrays");
    if (t < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return fail(DMTS_ERR_ARG, "need t >= 1, lr > 0, 0 <= beta < 1, eps > 0");
    const size_t n = m.n_params;
    std::vector<double> g(n);
    if (is_device_ptr(grad)) CUDA_TRY(cudaMemcpy(g.data(), grad, sizeof(double) * n, cudaMemcpyDeviceToHost));
    else std::copy(grad, grad + n, g.begin());
    const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    std::vector<double> th = m.hp;
    for (size_t k = 0; k < n; ++k) {
        if (!isfinite(g[k])) return fail(DMTS_ERR_ARG, "gradient entry %zu is not finite", k);
        m1[k] = beta1 * m1[k] + (1.0 - beta1) * g[k];
        m2[k] = beta2 * m2[k] + (1.0 - beta2) * g[k] * g[k];
        th[k] -= lr * (m1[k] / c1) / (sqrt(m2[k] / c2) + eps);
    }
    LaunchScope ls(c);
    int rc = upload_params(c, m, th.data());
    if (rc) return rc;
    if ((rc = prepare_embedding(c, m))) return rc;
    c->forces_valid = false;
    return sync_check(c);
}

int dmts_time_stages(dmts_ctx* c, int which, int reps, double* ms_out, int n_out) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_time_stages");
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    if (!c->m[which].present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (!c->state_set) return fail(DMTS_ERR_STATE, "no state set");
    if (reps < 1 || !ms_out) return fail(DMTS_ERR_ARG, "reps must be >= 1 and ms_out non-NULL");
    LaunchScope ls(c);
    const int n_st = 3 + 4 * c->m[which].L;
    if (n_out < n_st) return fail(DMTS_ERR_ARG, "ms_out needs %d entries", n_st);
    std::vector<double> acc;
    int rc = time_stages_impl(c, which, reps, acc);
    if (rc) return rc;
    for (int k = 0; k < n_st; ++k) ms_out[k] = acc[k];
    return n_st;
}

}  // extern "C"

namespace {

// Per-stage milliseconds of one evaluation of model `which` (CUDA events on
// the context's stream, mean over reps), in the order of dmts_time_stages.
int time_stages_impl(dmts_ctx* c, int which, int reps, std::vector<double>& acc) {
    Model& m = c->m[which];
    const int L = m.L;
    const int n_st = 3 + 4 * L;
    int rc;
    // one untimed evaluation sizes the capacities
    if ((rc = reset_flags(c))) return rc;
    enqueue_eval(c, which, true);
    if ((rc = sync_check(c))) return rc;
    if (c->h_flags[kFlagOverflow]) {
        if ((rc = grow_capacity(c))) return rc;
        if ((rc = reset_flags(c))) return rc;
        enqueue_eval(c, which, true);
        if ((rc = sync_check(c))) return rc;
    }
    cudaStream_t s = c->stream;
    std::vector<cudaEvent_t> ev(2 * n_st);
    for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
    acc.assign(n_st, 0.0);
    // stages without work (the embedding, built once per parameter upload, and
    // the layer-0 per-atom adjoint) are not timed: they read 0
    std::vector<char> timed(n_st, 1);
    timed[1] = 0;
    timed[2 + 3 * L] = 0;
    for (int r = 0; r < reps; ++r) {
        auto begin = [&](int slot) { cudaEventRecord(ev[2 * slot], s); };
        auto end = [&](int slot) { cudaEventRecord(ev[2 * slot + 1], s); };
        begin(0);
        enqueue_neighbors(c, which, true);
        end(0);
        PotArgs a = pot_args(c, m);
        for (int l = 0; l < L; ++l) {
            PotArgs f = fwd_args(c, a, m, l);
            begin(2 + l);
            launch_edge_fwd(c, m, f);
            end(2 + l);
            begin(2 + L + l);
            launch_atom_fwd_m(c, m, f);
            end(2 + L + l);
        }
        for (int l = L - 1; l >= 0; --l) {
            PotArgs b = bwd_args(a, m, l);
            begin(2 + 2 * L + l);
            launch_edge_bwd(c, m, b);
            end(2 + 2 * L + l);
            if (l > 0) {
                begin(2 + 3 * L + l);
                launch_atom_bwd_m(c, m, b);
                end(2 + 3 * L + l);
            }
        }
        begin(2 + 4 * L);
        launch_system_sum(c->n_sys, c->d_off, m.Ei, m.E, 1, m.esum, s);
        end(2 + 4 * L);
        CUDA_TRY(cudaEventSynchronize(ev[2 * n_st - 1]));
        for (int q = 0; q < n_st; ++q) {
            if (!timed[q]) continue;
            float t = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]));
            acc[q] += t;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int k = 0; k < n_st; ++k) acc[k] /= reps;
    return sync_check(c);
}

}  // namespace

extern "C" {

long long dmts_launch_count(dmts_ctx* c) { return c ? c->launches : -1; }

int dmts_monitor(dmts_ctx* c, double* max_df, long long* n_fallback, long long* n_flagged, long long* hist,
                 int n_bins) {
    CTX_GUARD(c);
    ForceMonitor m{};
    CUDA_TRY(cudaMemcpyAsync(&m, c->d_mon, sizeof(m), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (max_df) memcpy(max_df, &m.max_bits, sizeof(double));
    if (n_fallback) *n_fallback = (long long)m.n_fallback;
    if (n_flagged) *n_flagged = (long long)m.n_flagged;
    if (hist)
        for (int b = 0; b < n_bins && b < kMonitorBins; ++b) hist[b] = (long long)m.hist[b];
    return kMonitorBins;
}

int dmts_monitor_reset(dmts_ctx* c) {
    CTX_GUARD(c);
    CUDA_TRY(cudaMemsetAsync(c->d_mon, 0, sizeof(ForceMonitor), c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->fallback_seen = 0;
    return DMTS_OK;
}

int dmts_hmr_masses(int n_atoms, const double* mass, int n_bonds, const int* bonds, double h_mass,
                    double* mass_out) {
    g_err.clear();
    if (n_atoms < 0 || n_bonds < 0) return fail(DMTS_ERR_ARG, "negative count");
    if ((n_atoms > 0 && (!mass || !mass_out)) || (n_bonds > 0 && !bonds)) return fail(DMTS_ERR_ARG, "NULL array");
    if (!(h_mass > 0.0) || !isfinite(h_mass)) return fail(DMTS_ERR_ARG, "h_mass must be > 0");
    const double h_max = 1.5;                      // hydrogens: atoms lighter than 1.5 amu
    std::vector<double> m(mass, mass + n_atoms);
    std::vector<char> moved(n_atoms, 0);
    for (int b = 0; b < n_bonds; ++b) {
        const int a0 = bonds[2 * b], a1 = bonds[2 * b + 1];
        if (a0 < 0 || a0 >= n_atoms || a1 < 0 || a1 >= n_atoms) return fail(DMTS_ERR_ARG, "bond %d out of range", b);
        for (int side = 0; side < 2; ++side) {
            const int h = side ? a1 : a0, heavy = side ? a0 : a1;
            if (mass[h] < h_max && mass[heavy] >= h_max && !moved[h]) {
                m[heavy] -= h_mass - mass[h];
                m[h] = h_mass;
                moved[h] = 1;
            }
        }
    }
    for (int i = 0; i < n_atoms; ++i)
        if (!(m[i] > 0.0)) return fail(DMTS_ERR_ARG, "repartitioning leaves atom %d with mass %g", i, m[i]);
    std::copy(m.begin(), m.end(), mass_out);
    return DMTS_OK;
}

int dmts_neighbor_stats(dmts_ctx* c, long long* n_checks, long long* n_rebuilds) {
    CTX_GUARD(c);
    VerletState st{};
    if (c->skin > 0) {
        CUDA_TRY(cudaMemcpyAsync(&st, c->d_vl, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    if (n_checks) *n_checks = st.n_checks;
    if (n_rebuilds) *n_rebuilds = st.n_rebuilds;
    return DMTS_OK;
}

int dmts_get_tuning(dmts_ctx* c, int which, int* atoms_fwd, int* atoms_bwd) {
    if (!c) return fail(DMTS_ERR_ARG, "context is NULL");
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    if (!c->m[which].present) return fail(DMTS_ERR_ARG, "no small model in this context");
    const bool tc = c->m[which].precision == DMTS_BF16_MLP;
    if (atoms_fwd) *atoms_fwd = tc ? c->m[which].cps_fwd : c->m[which].apc_fwd;
    if (atoms_bwd) *atoms_bwd = tc ? c->m[which].cps_bwd : c->m[which].apc_bwd;
    return c->tuned ? 1 : 0;
}

int dmts_set_tuning(dmts_ctx* c, int which, int fwd, int bwd, int bwd_tiles) {
    CTX_GUARD(c);
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    Model& m = c->m[which];
    if (!m.present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (fwd < 1 || bwd < 1) return fail(DMTS_ERR_ARG, "granularity must be >= 1");
    if (bwd_tiles < 0 || bwd_tiles > 2) return fail(DMTS_ERR_ARG, "bwd_tiles must be 0, 1 or 2");
    if (m.precision == DMTS_BF16_MLP) {
        if (bwd_tiles > 0) m.bwd_tiles = bwd_tiles;
        m.cps_fwd = std::min(fwd, bf16_max_ctas_per_sm(m.F, false));
        m.cps_bwd = std::min(bwd, bf16_max_ctas_per_sm(m.F, true, m.bwd_tiles));
    } else {
        m.apc_fwd = std::min(fwd, max_atoms_per_cta_f32(m.F, m.K, false));
        m.apc_bwd = std::min(bwd, max_atoms_per_cta_f32(m.F, m.K, true));
    }
    c->tuned = true;                          // the tuner keeps the caller's choice
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return DMTS_OK;
}

int dmts_get_bwd_tiles(dmts_ctx* c, int which) {
    if (!c) return fail(DMTS_ERR_ARG, "context is NULL");
    if (which != DMTS_SMALL && which != DMTS_BIG) return fail(DMTS_ERR_ARG, "which must be 0 or 1");
    const Model& m = c->m[which];
    if (!m.present) return fail(DMTS_ERR_ARG, "no small model in this context");
    if (m.precision != DMTS_BF16_MLP) return 1;
    return m.bwd_tiles > 0 ? m.bwd_tiles : bf16_default_bwd_tiles(m.F);
}

int dmts_wait_selftest(dmts_ctx* c, int arrive, int max_polls) {
    CTX_GUARD(c);
    Range nvtx_range("dmts_wait_selftest");
    if (max_polls < 1 || max_polls > (1 << 22)) return fail(DMTS_ERR_ARG, "max_polls must be in [1, 2^22]");
    LaunchScope ls(c);
    int rc = reset_flags(c);
    if (rc) return rc;
    launch_wait_selftest(arrive ? 1 : 0, (unsigned int)max_polls, c->d_flags + kFlagTimeout, c->stream);
    const bool valid = c->forces_valid;       // the self-test touches no force or state
    rc = sync_check(c);
    if (!c->broken) c->forces_valid = valid;
    return rc;
}

int dmts_philox4x32_10(int n, const unsigned int* ctr, const unsigned int* key, unsigned int* out) {
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(DMTS_ERR_ARG, "bad arguments");
    if (n == 0) return DMTS_OK;
    uint4 *d_in = nullptr, *d_out = nullptr;
    CUDA_TRY(dalloc(&d_in, (size_t)n));
    cudaError_t e = dalloc(&d_out, (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(d_in, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_philox_words(n, d_in, key[0], key[1], d_out, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    dfree(d_in);
    dfree(d_out);
    if (e != cudaSuccess) return fail(DMTS_ERR_CUDA, "philox: %s", cudaGetErrorString(e));
    return DMTS_OK;
}

}  // extern "C"
