// Integrator kernels: the kicks and drifts of Algorithm 1 (thermostat: the
// identity, NVE, or the Langevin O-step) and of velocity Verlet (or BAOAB),
// on the FP64 SoA state, fused with periodic wrapping and the fixed-point
// quantisation that the next force evaluation reads. One thread per atom; every kernel streams x, v, 1/m and
// the FP32 forces once.
#include <algorithm>

#include "internal.cuh"

namespace dmts {

// 1 eV/(Angstrom amu) expressed in Angstrom/fs^2, and its inverse (1 amu
// (Angstrom/fs)^2 in eV): (1.602176634e-19 J / 1e-10 m) / 1.66053906660e-27 kg
// = 9.648533216e17 m/s^2.
constexpr double kAccel = 9.648533215665327e-3;
constexpr double kKinetic = 103.64269652680505;

// x - L floor(x / L) for periodic boxes; coordinates already inside [0, L)
// are returned as they are (the common case needs no FP64 division).
// Threads per CTA of the integrator kernels: their FP64 arithmetic (GB300
// issues FP64 at a small fraction of its FP32 rate) spreads over every SM
// only with small CTAs (192 of them for 12,288 atoms instead of 48).
constexpr int kIntThreads = 64;

int integrator_blocks(int n_atoms) { return (n_atoms + kIntThreads - 1) / kIntThreads; }

// The fused energy epilogue of a closing kernel (see EnergyFuse); every
// thread of every block calls it (ke_i = 0 past the last atom). Sums are
// FP64: within a block in warp order, then over the blocks in block order.
__device__ __forceinline__ void energy_epilogue(const EnergyFuse& ef, int n, int i, double ke_i, int* flags) {
    __shared__ double s_part[2][kIntThreads / 32];
    __shared__ bool s_last_e;
    double a = i < n ? ke_i : 0.0;
    double b = (i < n && ef.ei) ? ef.ei[i] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s_part[0][w] = a; s_part[1][w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { ta += s_part[0][k]; tb += s_part[1][k]; }
        ef.part[2 * blockIdx.x] = ta;
        ef.part[2 * blockIdx.x + 1] = tb;
        __threadfence();
        s_last_e = atomicAdd(ef.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last_e && w == 0) {
        __threadfence();
        double ua = 0.0, ub = 0.0;
        for (int k = lane; k < (int)gridDim.x; k += 32) {
            ua += __ldcg(ef.part + 2 * k);
            ub += __ldcg(ef.part + 2 * k + 1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ua += __shfl_down_sync(0xffffffffu, ua, o);
            ub += __shfl_down_sync(0xffffffffu, ub, o);
        }
        if (lane == 0) {
            *ef.ekin = ua;
            if (ef.ei) *ef.epot = ub;
            const double ep = *ef.epot;
            const int step = flags[kFlagStep];
            if (step < ef.ring_len) {
                double* o = ef.ring + (size_t)step * 3;
                o[0] = ep;
                o[1] = ua;
                o[2] = ep + ua;
            }
            flags[kFlagStep] = step + 1;
            *ef.ticket = 0u;
        }
    }
}

__device__ __forceinline__ double wrap_coord(double x, double L) {
    return (L > 0.0 && (x < 0.0 || x >= L)) ? x - L * floor(x / L) : x;
}

// Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC 2011): per
// round, words 0 and 2 are multiplied by the two Philox multipliers, their
// high halves are crossed with words 1 and 3 and the key; the key advances by
// the two Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The generator's raw output for given counters and one key: the words the
// thermostat's noise is made of, for comparison with published test vectors.
__global__ void k_philox_words(int n, const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1,
                               uint4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

// Three standard normals for atom i at inner step t: uniforms (w + 1/2) 2^-32
// of the four Philox words, Box-Muller on (u0, u1) for two and on (u2, u3)
// for the third.
__device__ __forceinline__ void langevin_normals(unsigned int i, unsigned long long t, uint32_t k0, uint32_t k1,
                                                 double* n) {
    const uint4 w = philox4x32_10(make_uint4(i, (unsigned int)t, (unsigned int)(t >> 32), 0u), k0, k1);
    const double s32 = 2.3283064365386963e-10;          // 2^-32
    const double u0 = ((double)w.x + 0.5) * s32, u1 = ((double)w.y + 0.5) * s32;
    const double u2 = ((double)w.z + 0.5) * s32, u3 = ((double)w.w + 0.5) * s32;
    const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    n[0] = r01 * cs;
    n[1] = r01 * sn;
    n[2] = r23 * cospi(2.0 * u3);
}

__device__ __forceinline__ unsigned int fixed_of(double v, double o, double inv) {
    long long k = (long long)floor((v - o) * inv);
    return (unsigned int)(k & 0xffffffffll);
}

__global__ void k_set_state(int n, const double* __restrict__ xa, const double* __restrict__ va,
                            const int* __restrict__ sys, const double* __restrict__ box,
                            double* __restrict__ x, double* __restrict__ v, int* __restrict__ moved) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double L = box[sys[i]];
    bool diff = false;
    for (int c = 0; c < 3; ++c) {
        const double w = wrap_coord(xa[3 * (size_t)i + c], L);
        if (moved) diff = diff || __double_as_longlong(w) != __double_as_longlong(x[(size_t)c * n + i]);
        x[(size_t)c * n + i] = w;
        v[(size_t)c * n + i] = va ? va[3 * (size_t)i + c] : 0.0;
    }
    if (diff) atomicOr(moved, 1);
}

void launch_philox_words(int n, const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, cudaStream_t s) {
    if (n <= 0) return;
    k_philox_words<<<(n + 255) / 256, 256, 0, s>>>(n, ctr, k0, k1, out);
    count_launch();
}

void launch_set_state(int n_atoms, const double* x_aos, const double* v_aos, const int* sys_of_atom,
                      const double* box, double* x, double* v, int* moved, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_set_state<<<(n_atoms + 255) / 256, 256, 0, s>>>(n_atoms, x_aos, v_aos, sys_of_atom, box, x, v, moved);
    count_launch();
}

__global__ void k_get_state(int n, const double* __restrict__ x, const double* __restrict__ v,
                            double* __restrict__ xa, double* __restrict__ va) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 3; ++c) {
        if (xa) xa[3 * (size_t)i + c] = x[(size_t)c * n + i];
        if (va) va[3 * (size_t)i + c] = v[(size_t)c * n + i];
    }
}

void launch_get_state(int n_atoms, const double* x, const double* v, double* x_aos, double* v_aos,
                      cudaStream_t s) {
    if (n_atoms == 0) return;
    k_get_state<<<(n_atoms + 255) / 256, 256, 0, s>>>(n_atoms, x, v, x_aos, v_aos);
    count_launch();
}

__global__ void k_forces_out(int n, const float* __restrict__ f, double* __restrict__ fa) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 3; ++c) fa[3 * (size_t)i + c] = (double)f[(size_t)c * n + i];
}

void launch_forces_out(int n_atoms, const float* f, double* f_aos, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_forces_out<<<(n_atoms + 255) / 256, 256, 0, s>>>(n_atoms, f, f_aos);
    count_launch();
}

// Algorithm 1, inner step before the small force:
//   first:  v += (dt/2m) (F - F_small)        (outer half-kick)
//   else:   v += (h/2m) F_small               (post-kick of the previous inner step)
//   then    v += (h/2m) F_small; x += (h/2) v; [thermo = identity]; x += (h/2) v
// with the position wrapped after each half-drift; then quantise x, and put
// the atom into the fixed-capacity cells of the models evaluated next (cp0,
// cp1; nc = 0: none), as the pair-list build would.
// Atom i's small-model force (see ForceFold): split rows summed from the
// tiles' carry slots (head tile's last slot, then the later tiles' first
// slots, in tile order, in FP32), rows without pairs zero, other rows read
// from fs. Returns true if the value did not come from fs.
__device__ __forceinline__ bool folded_force(const ForceFold& ff, const float* fs, int n, int i, float f[3]) {
    if (ff.row_ptr) {
        const long long r0 = min((long long)ff.row_ptr[i], ff.e_cap), r1 = min((long long)ff.row_ptr[i + 1], ff.e_cap);
        if (r1 <= r0) {
            f[0] = f[1] = f[2] = 0.f;
            return true;
        }
        const long long t0 = r0 >> 7, t1 = (r1 - 1) >> 7;
        if (t0 != t1) {
            const float* cl = ff.carry + (2 * t0 + 1) * (long long)ff.carry_w + ff.F;
#pragma unroll
            for (int c = 0; c < 3; ++c) f[c] = cl[c];
            for (long long u = t0 + 1; u <= t1; ++u) {
                const float* cf = ff.carry + 2 * u * (long long)ff.carry_w + ff.F;
#pragma unroll
                for (int c = 0; c < 3; ++c) f[c] += cf[c];
            }
            return true;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = fs[(size_t)c * n + i];
    return false;
}

__global__ void k_respa_pre(int n, int first, double c_outer, double c_inner, double half_h,
                            double* __restrict__ x, double* __restrict__ v,
                            const double* __restrict__ inv_m, const float* __restrict__ fs,
                            const float* __restrict__ fb, const int* __restrict__ sys,
                            const double* __restrict__ box, const Frame* __restrict__ frame,
                            uint4* __restrict__ q, int* __restrict__ flags, VerletCheck vc, Langevin lg,
                            CellPlace cp0, CellPlace cp1, ForceFold fold) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (i < n) {
        int s = sys[i];
        double L = box[s];
        Frame fr = frame[s];
        double im = inv_m[i];
        unsigned int qc[3];
        bool ok = true;
        double xi[3] = {0.0, 0.0, 0.0}, sig = 0.0;
        if (lg.on) {
            langevin_normals((unsigned int)i, *lg.step + (unsigned long long)lg.offset, lg.key0, lg.key1, xi);
            sig = lg.c2 * sqrt(lg.kT_accel * im);
        }
        float fsi[3];
        (void)folded_force(fold, fs, n, i, fsi);
        for (int c = 0; c < 3; ++c) {
            size_t o = (size_t)c * n + i;
            double vv = v[o];
            double Fs = (double)fsi[c];
            if (first) vv = vv + c_outer * im * ((double)fb[o] - Fs);
            else vv = vv + c_inner * im * Fs;
            vv = vv + c_inner * im * Fs;
            double xx = wrap_coord(x[o] + half_h * vv, L);
            if (lg.on) vv = lg.c1 * vv + sig * xi[c];            // v <- thermo(v, h)
            xx = wrap_coord(xx + half_h * vv, L);
            ok = ok && isfinite(vv) && isfinite(xx);
            v[o] = vv;
            x[o] = xx;
            double oc = c == 0 ? fr.ox : (c == 1 ? fr.oy : fr.oz);
            qc[c] = fixed_of(xx, oc, fr.inv);
        }
        const uint4 qi = make_uint4(qc[0], qc[1], qc[2], (unsigned int)s);
        q[i] = qi;
        if (cp0.nc > 0) place_in_cell(cp0, i, qi, flags);
        if (cp1.nc > 0) place_in_cell(cp1, i, qi, flags);
        if (!ok) atomicOr(&flags[kFlagNonfinite], 1);
        if (vc.st) m = vl_disp2(x, vc.xref, (size_t)n, (size_t)i, L, vc.thr2);
    }
    if (vc.st) vl_block_decide(m, vc);               // the neighbour-list check of the new positions
}

void launch_respa_pre(int n_atoms, int first, double c_outer, double c_inner, double half_h,
                      double* x, double* v, const double* inv_mass, const float* f_small,
                      const float* f_big, const int* sys_of_atom, const double* box,
                      const Frame* frame, uint4* q, int* flags, const VerletCheck& vc,
                      const Langevin& lg, const CellPlace& cp0, const CellPlace& cp1,
                      const ForceFold& fold, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_respa_pre<<<(n_atoms + kIntThreads - 1) / kIntThreads, kIntThreads, 0, s>>>(n_atoms, first, c_outer, c_inner, half_h, x, v,
                                                     inv_mass, f_small, f_big, sys_of_atom, box,
                                                     frame, q, flags, vc, lg, cp0, cp1, fold);
    count_launch();
}

// After the big force: v += (h/2m) F_small (last inner post-kick), then
// v += (dt/2m) (F - F_small) (outer half-kick); per-atom kinetic energy.
// With a monitor: per-atom |F - F_small| (the forces of the step's end),
// reduced per block (maximum, atoms above the threshold, histogram) and
// over blocks; the last block to finish decides whether the step falls back
// (some atom above the threshold) and sets the graph conditional.
__global__ void __launch_bounds__(256) k_respa_post(int n, double c_outer, double c_inner, double* __restrict__ v,
                                                    const double* __restrict__ inv_m, float* fs,
                                                    const float* __restrict__ fb, const double* __restrict__ x,
                                                    double* __restrict__ ke, const double* __restrict__ mass,
                                                    int* __restrict__ flags, unsigned long long* __restrict__ step,
                                                    int advance, MonitorArgs mon, ForceFold fold, EnergyFuse ef) {
    __shared__ unsigned int s_hist[kMonitorBins];
    __shared__ double s_max[8];
    __shared__ unsigned int s_flag;
    __shared__ bool s_last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (mon.mon) {
        for (int b = threadIdx.x; b < kMonitorBins; b += blockDim.x) s_hist[b] = 0u;
        if (threadIdx.x == 0) s_flag = 0u;
        __syncthreads();
    }
    double df = 0.0, ke_i = 0.0;
    if (i < n) {
        if (step && i == 0) *step += (unsigned long long)advance;   // every reader of it ran in earlier kernels
        double im = inv_m[i];
        double v2 = 0.0, d2 = 0.0;
        bool ok = true;
        float fsi[3];
        if (folded_force(fold, fs, n, i, fsi))                  // complete the array for later readers
            for (int c = 0; c < 3; ++c) fs[(size_t)c * n + i] = fsi[c];
        for (int c = 0; c < 3; ++c) {
            size_t o = (size_t)c * n + i;
            double Fs = (double)fsi[c];
            const double dF = (double)fb[o] - Fs;
            d2 += dF * dF;
            double vv = v[o] + c_inner * im * Fs;
            vv = vv + c_outer * im * dF;
            v[o] = vv;
            v2 += vv * vv;
            ok = ok && isfinite(vv) && isfinite(x[o]);
        }
        ke_i = 0.5 * mass[i] * v2 * kKinetic;
        ke[i] = ke_i;
        if (!ok) atomicOr(&flags[kFlagNonfinite], 1);
        df = sqrt(d2);
        if (mon.mon) {
            int b = 0;
            if (df > 0.0) b = (int)floor((log10(df) + 3.0) * 8.0);
            b = b < 0 ? 0 : (b >= kMonitorBins ? kMonitorBins - 1 : b);
            if (!(df == df)) b = kMonitorBins - 1;                  // NaN: the top bin
            atomicAdd(&s_hist[b], 1u);
            if (mon.threshold > 0.0 && !(df <= mon.threshold)) atomicAdd(&s_flag, 1u);
        }
    }
    if (ef.on) energy_epilogue(ef, n, i, ke_i, flags);
    if (!mon.mon) return;
    if (!(df == df)) df = 1e300;
    double m = df;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, s_max[k]);
        const unsigned long long bits = (unsigned long long)__double_as_longlong(m);
        atomicMax(&mon.mon->max_bits, bits);
        atomicMax(&mon.mon->step_max_bits, bits);
        if (s_flag) atomicAdd(&mon.mon->n_flagged, (unsigned long long)s_flag);
    }
    for (int b = threadIdx.x; b < kMonitorBins; b += blockDim.x)
        if (s_hist[b]) atomicAdd(&mon.mon->hist[b], (unsigned long long)s_hist[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&mon.mon->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const double mx = __longlong_as_double((long long)atomicAdd(&mon.mon->step_max_bits, 0ull));
        const int fall = (mon.threshold > 0.0 && !(mx <= mon.threshold)) ? 1 : 0;
        mon.mon->n_fallback += (unsigned long long)fall;
        mon.mon->step_max_bits = 0ull;
        mon.mon->done = 0u;
        if (mon.use_cond) cudaGraphSetConditional(mon.cond, (unsigned int)fall);
    }
}

void launch_respa_post(int n_atoms, double c_outer, double c_inner, double* v,
                       const double* inv_mass, float* f_small, const float* f_big,
                       const double* x, double* ke, const double* mass, int* flags,
                       unsigned long long* step, int advance, const MonitorArgs& mon,
                       const ForceFold& fold, const EnergyFuse& ef, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_respa_post<<<(n_atoms + kIntThreads - 1) / kIntThreads, kIntThreads, 0, s>>>(n_atoms, c_outer, c_inner, v, inv_mass, f_small,
                                                      f_big, x, ke, mass, flags, step, advance, mon, fold, ef);
    count_launch();
}

__global__ void k_copy_state(int n, const double* __restrict__ x, const double* __restrict__ v,
                             const float* __restrict__ f, double* __restrict__ xo, double* __restrict__ vo,
                             float* __restrict__ fo) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * n; t += gridDim.x * blockDim.x) {
        xo[t] = x[t];
        vo[t] = v[t];
        fo[t] = f[t];
    }
}

void launch_copy_state(int n_atoms, const double* x, const double* v, const float* f, double* x_out,
                       double* v_out, float* f_out, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_copy_state<<<std::min(4 * 152, (3 * n_atoms + 255) / 256), 256, 0, s>>>(n_atoms, x, v, f, x_out, v_out, f_out);
    count_launch();
}

// Velocity Verlet: v += (dt/2m) F; x += dt v (wrapped); quantise.
__global__ void k_vv_pre(int n, double c_half, double dt, double* __restrict__ x,
                         double* __restrict__ v, const double* __restrict__ inv_m,
                         const float* __restrict__ f, const int* __restrict__ sys,
                         const double* __restrict__ box, const Frame* __restrict__ frame,
                         uint4* __restrict__ q, int* __restrict__ flags, VerletCheck vc, Langevin lg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (i < n) {
        int s = sys[i];
        double L = box[s];
        Frame fr = frame[s];
        double im = inv_m[i];
        unsigned int qc[3];
        bool ok = true;
        double xi[3] = {0.0, 0.0, 0.0}, sig = 0.0;
        if (lg.on) {
            langevin_normals((unsigned int)i, *lg.step + (unsigned long long)lg.offset, lg.key0, lg.key1, xi);
            sig = lg.c2 * sqrt(lg.kT_accel * im);
        }
        for (int c = 0; c < 3; ++c) {
            size_t o = (size_t)c * n + i;
            double vv = v[o] + c_half * im * (double)f[o];
            double xx;
            if (lg.on) {                                            // BAOAB: A, O, A
                xx = wrap_coord(x[o] + (0.5 * dt) * vv, L);
                vv = lg.c1 * vv + sig * xi[c];
                xx = wrap_coord(xx + (0.5 * dt) * vv, L);
            } else {
                xx = wrap_coord(x[o] + dt * vv, L);
            }
            ok = ok && isfinite(vv) && isfinite(xx);
            v[o] = vv;
            x[o] = xx;
            double oc = c == 0 ? fr.ox : (c == 1 ? fr.oy : fr.oz);
            qc[c] = fixed_of(xx, oc, fr.inv);
        }
        q[i] = make_uint4(qc[0], qc[1], qc[2], (unsigned int)s);
        if (!ok) atomicOr(&flags[kFlagNonfinite], 1);
        if (vc.st) m = vl_disp2(x, vc.xref, (size_t)n, (size_t)i, L, vc.thr2);
    }
    if (vc.st) vl_block_decide(m, vc);
}

void launch_vv_pre(int n_atoms, double c_half, double dt, double* x, double* v,
                   const double* inv_mass, const float* f, const int* sys_of_atom,
                   const double* box, const Frame* frame, uint4* q, int* flags, const VerletCheck& vc,
                   const Langevin& lg, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_vv_pre<<<(n_atoms + kIntThreads - 1) / kIntThreads, kIntThreads, 0, s>>>(n_atoms, c_half, dt, x, v, inv_mass, f, sys_of_atom,
                                                  box, frame, q, flags, vc, lg);
    count_launch();
}

__global__ void k_vv_post(int n, double c_half, double* __restrict__ v,
                          const double* __restrict__ inv_m, const float* __restrict__ f,
                          const double* __restrict__ x, double* __restrict__ ke,
                          const double* __restrict__ mass, int* __restrict__ flags,
                          unsigned long long* __restrict__ step, EnergyFuse ef) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke_i = 0.0;
    if (i < n) {
        if (step && i == 0) *step += 1ull;
        double im = inv_m[i];
        double v2 = 0.0;
        bool ok = true;
        for (int c = 0; c < 3; ++c) {
            size_t o = (size_t)c * n + i;
            double vv = v[o] + c_half * im * (double)f[o];
            v[o] = vv;
            v2 += vv * vv;
            ok = ok && isfinite(vv) && isfinite(x[o]);
        }
        ke_i = 0.5 * mass[i] * v2 * kKinetic;
        ke[i] = ke_i;
        if (!ok) atomicOr(&flags[kFlagNonfinite], 1);
    }
    if (ef.on) energy_epilogue(ef, n, i, ke_i, flags);
}

void launch_vv_post(int n_atoms, double c_half, double* v, const double* inv_mass,
                    const float* f, const double* x, double* ke, const double* mass, int* flags,
                    unsigned long long* step, const EnergyFuse& ef, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_vv_post<<<(n_atoms + kIntThreads - 1) / kIntThreads, kIntThreads, 0, s>>>(n_atoms, c_half, v, inv_mass, f, x, ke,
                                                                               mass, flags, step, ef);
    count_launch();
}

__global__ void k_energy_record(int n_sys, const double* __restrict__ ep, const double* __restrict__ ek,
                                double* __restrict__ ring, int ring_len, int* __restrict__ flags) {
    int step = flags[kFlagStep];
    for (int s = threadIdx.x; s < n_sys; s += blockDim.x) {
        if (step < ring_len) {
            double* o = ring + ((size_t)step * n_sys + s) * 3;
            o[0] = ep[s];
            o[1] = ek[s];
            o[2] = ep[s] + ek[s];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) flags[kFlagStep] = step + 1;
}

void launch_energy_record(int n_sys, const double* epot, const double* ekin, double* ring,
                          int ring_len, int* flags, cudaStream_t s) {
    k_energy_record<<<1, 256, 0, s>>>(n_sys, epot, ekin, ring, ring_len, flags);
    count_launch();
}

double accel_constant() { return kAccel; }

}  // namespace dmts
