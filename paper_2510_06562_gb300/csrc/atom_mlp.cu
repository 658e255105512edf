// Per-atom MLPs of the potential (FP32, register-blocked SIMT), used by both
// precisions after the edge passes have produced the per-atom sums:
//
//   forward, layer l:   z = m U1 + c1;  h <- h + SiLU(z) U2 + c2;
//                       l < L-1:  u^{l+1} = h W_in^{l+1}
//                       l = L-1:  q = h R1 + d1;  E_i = SiLU(q) . R2 + d2 + e0[Z_i] + E_rep,i
//                                 and the first adjoint steps:
//                                 gh = (SiLU'(q) * R2) R1^T;  mbar^l = ((gh U2^T) * SiLU'(z)) U1^T
//   backward, layer l >= 1:  gh <- gh + ubar^l W_in^{l T};
//                            mbar^{l-1} = ((gh U2^{l-1 T}) * SiLU'(z^{l-1})) U1^{l-1 T}
//
// A CTA of 256 threads takes A = 4096 / F atoms; every stage is an
// [A x F] x [F x F] product with each thread owning 4 atoms x 4 features,
// the input kept transposed in shared memory ([k][atom]) and the weight
// matrix staged as W[k][f] (or its transpose).
#include "internal.cuh"

namespace dmts {

namespace {

constexpr int kAT = 256;

template <int F>
struct AtomTile {
    static constexpr int A = 4096 / F;      // atoms per CTA
    static constexpr int AG = A / 4;        // atom groups
    static constexpr int FG = F / 4;        // feature groups
    static constexpr int IS = A + 4;        // row stride of transposed inputs [k][a]
    static constexpr int WS = F + 4;        // row stride of staged weights [k][f]
    static_assert(AG * FG == kAT, "tile");
};

__device__ __forceinline__ float sig(float x) { return 1.0f / (1.0f + __expf(-x)); }

template <int F>
__device__ __forceinline__ void load_w(float* Ws, const float* __restrict__ W, bool transpose) {
    using T = AtomTile<F>;
    __syncthreads();
    for (int t = threadIdx.x; t < F * F; t += kAT) {
        int r = t / F, c = t % F;            // W[r][c], row-major
        if (transpose) Ws[c * T::WS + r] = __ldg(W + t);
        else Ws[r * T::WS + c] = __ldg(W + t);
    }
    __syncthreads();
}

// acc[a][f] = sum_k inT[k][a0 + a] * Ws[k][f0 + f]
template <int F>
__device__ __forceinline__ void gemm4x4(const float* inT, const float* Ws, int a0, int f0, float acc[4][4]) {
    using T = AtomTile<F>;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int f = 0; f < 4; ++f) acc[a][f] = 0.f;
#pragma unroll 8
    for (int k = 0; k < F; ++k) {
        float4 x = *reinterpret_cast<const float4*>(inT + k * T::IS + a0);
        float4 w = *reinterpret_cast<const float4*>(Ws + k * T::WS + f0);
        float xa[4] = {x.x, x.y, x.z, x.w}, wf[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int f = 0; f < 4; ++f) acc[a][f] += xa[a] * wf[f];
    }
}

// Store v[a][f] transposed into outT[k = f][a].
template <int F>
__device__ __forceinline__ void store_t(float* outT, int a0, int f0, const float v[4][4]) {
    using T = AtomTile<F>;
#pragma unroll
    for (int f = 0; f < 4; ++f)
        *reinterpret_cast<float4*>(outT + (f0 + f) * T::IS + a0) = make_float4(v[0][f], v[1][f], v[2][f], v[3][f]);
}

// Load rows [atom][F] of a global [N][F] array into inT (transposed), zero past N.
template <int F>
__device__ __forceinline__ void load_rows_t(float* inT, const float* __restrict__ src, int base, int n_atoms) {
    using T = AtomTile<F>;
    for (int t = threadIdx.x; t < T::A * F; t += kAT) {
        int a = t / F, f = t % F;
        int i = base + a;
        inT[f * T::IS + a] = i < n_atoms ? src[(size_t)i * F + f] : 0.f;
    }
}

template <int F>
__device__ __forceinline__ void store_rows(float* __restrict__ dst, int base, int n_atoms, int a0, int f0,
                                           const float v[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int i = base + a0 + a;
        if (i < n_atoms)
            *reinterpret_cast<float4*>(dst + (size_t)i * F + f0) = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
    }
}

template <int F>
__device__ __forceinline__ void load_rows4(float v[4][4], const float* __restrict__ src, int base, int n_atoms,
                                           int a0, int f0) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int i = base + a0 + a;
        float4 x = i < n_atoms ? *reinterpret_cast<const float4*>(src + (size_t)i * F + f0) : make_float4(0, 0, 0, 0);
        v[a][0] = x.x; v[a][1] = x.y; v[a][2] = x.z; v[a][3] = x.w;
    }
}

template <int F>
__global__ void __launch_bounds__(kAT) k_atom_fwd(PotArgs p, const float* __restrict__ msg) {
    using T = AtomTile<F>;
    extern __shared__ float4 smem4[];
    float* X = reinterpret_cast<float*>(smem4);      // [F][IS]
    float* Y = X + F * T::IS;                        // [F][IS]
    float* Ws = Y + F * T::IS;                       // [F][WS]
    __shared__ float sE[T::A];
    const int l = p.layer;
    const int base = blockIdx.x * T::A;
    const int tid = threadIdx.x, fg = tid % T::FG, ag = tid / T::FG;
    const int f0 = 4 * fg, a0 = 4 * ag;
    const float* P = p.P;
    const bool last = (l == p.n_layers - 1);
    float z[4][4], v[4][4], h[4][4];

    load_rows_t<F>(X, msg, base, p.n_atoms);
    load_w<F>(Ws, P + p.off.U1[l], false);
    gemm4x4<F>(X, Ws, a0, f0, z);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float c1 = __ldg(P + p.off.c1[l] + f0 + f);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            z[a][f] += c1;
            v[a][f] = z[a][f] * sig(z[a][f]);
        }
    }
    store_rows<F>(p.z, base, p.n_atoms, a0, f0, z);
    store_t<F>(Y, a0, f0, v);
    load_w<F>(Ws, P + p.off.U2[l], false);
    gemm4x4<F>(Y, Ws, a0, f0, v);
    load_rows4<F>(h, p.h, base, p.n_atoms, a0, f0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float c2 = __ldg(P + p.off.c2[l] + f0 + f);
#pragma unroll
        for (int a = 0; a < 4; ++a) h[a][f] += v[a][f] + c2;
    }
    store_rows<F>(p.h, base, p.n_atoms, a0, f0, h);
    store_t<F>(X, a0, f0, h);
    if (!last) {
        load_w<F>(Ws, P + p.off.W_in[l + 1], false);
        gemm4x4<F>(X, Ws, a0, f0, v);
        store_rows<F>(p.u_next, base, p.n_atoms, a0, f0, v);
        return;
    }
    // readout and its adjoint
    load_w<F>(Ws, P + p.off.R1, false);
    gemm4x4<F>(X, Ws, a0, f0, v);
    float e_part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float d1 = __ldg(P + p.off.d1 + f0 + f), r2 = __ldg(P + p.off.R2 + f0 + f);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float q = v[a][f] + d1;
            float s = sig(q);
            e_part[a] += q * s * r2;
            v[a][f] = s * (1.f + q * (1.f - s)) * r2;     // dE/dq
        }
    }
    // sum the energy terms over the FG threads of this atom group (consecutive lanes)
#pragma unroll
    for (int a = 0; a < 4; ++a)
        for (int o = T::FG / 2; o > 0; o >>= 1) e_part[a] += __shfl_xor_sync(0xffffffffu, e_part[a], o);
    if (fg == 0)
        for (int a = 0; a < 4; ++a) sE[a0 + a] = e_part[a];
    store_t<F>(Y, a0, f0, v);
    load_w<F>(Ws, P + p.off.R1, true);
    gemm4x4<F>(Y, Ws, a0, f0, v);                    // gh = gq R1^T
    store_rows<F>(p.gh, base, p.n_atoms, a0, f0, v);
    store_t<F>(X, a0, f0, v);
    for (int a = tid; a < T::A; a += kAT) {
        int i = base + a;
        if (i < p.n_atoms)
            p.Ei[i] = (double)sE[a] + (double)__ldg(P + p.off.d2) + (double)__ldg(P + p.off.e0 + p.species[i]) +
                      (double)p.erep[i];
    }
    load_w<F>(Ws, P + p.off.U2[l], true);
    gemm4x4<F>(X, Ws, a0, f0, v);                    // gy = gh U2^T
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            float s = sig(z[a][f]);
            v[a][f] *= s * (1.f + z[a][f] * (1.f - s));
        }
    store_t<F>(Y, a0, f0, v);
    load_w<F>(Ws, P + p.off.U1[l], true);
    gemm4x4<F>(Y, Ws, a0, f0, v);                    // mbar = gz U1^T
    store_rows<F>(p.mbar_out, base, p.n_atoms, a0, f0, v);
}

template <int F>
__global__ void __launch_bounds__(kAT) k_atom_bwd(PotArgs p, const float* __restrict__ ubar) {
    using T = AtomTile<F>;
    extern __shared__ float4 smem4[];
    float* X = reinterpret_cast<float*>(smem4);
    float* Y = X + F * T::IS;
    float* Ws = Y + F * T::IS;
    const int l = p.layer;   // >= 1
    const int base = blockIdx.x * T::A;
    const int tid = threadIdx.x, fg = tid % T::FG, ag = tid / T::FG;
    const int f0 = 4 * fg, a0 = 4 * ag;
    const float* P = p.P;
    float v[4][4], g[4][4], z[4][4];
    load_rows_t<F>(X, ubar, base, p.n_atoms);
    load_w<F>(Ws, P + p.off.W_in[l], true);
    gemm4x4<F>(X, Ws, a0, f0, v);                    // ubar W_in^T
    load_rows4<F>(g, p.gh, base, p.n_atoms, a0, f0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int f = 0; f < 4; ++f) g[a][f] += v[a][f];
    store_rows<F>(p.gh, base, p.n_atoms, a0, f0, g);
    store_t<F>(Y, a0, f0, g);
    load_w<F>(Ws, P + p.off.U2[l - 1], true);
    gemm4x4<F>(Y, Ws, a0, f0, v);                    // gy = gh U2^T
    load_rows4<F>(z, p.z_prev, base, p.n_atoms, a0, f0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            float s = sig(z[a][f]);
            v[a][f] *= s * (1.f + z[a][f] * (1.f - s));
        }
    store_t<F>(X, a0, f0, v);
    load_w<F>(Ws, P + p.off.U1[l - 1], true);
    gemm4x4<F>(X, Ws, a0, f0, v);                    // mbar^{l-1} = gz U1^T
    store_rows<F>(p.mbar_out, base, p.n_atoms, a0, f0, v);
}

template <int F>
size_t atom_smem() {
    using T = AtomTile<F>;
    return sizeof(float) * (2 * F * T::IS + F * T::WS);
}

template <int F>
void atom_fwd_go(const PotArgs& p, const float* msg, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_atom_fwd<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)atom_smem<F>());
        attr = true;
    }
    int grid = (p.n_atoms + AtomTile<F>::A - 1) / AtomTile<F>::A;
    k_atom_fwd<F><<<grid, kAT, atom_smem<F>(), s>>>(p, msg);
}

template <int F>
void atom_bwd_go(const PotArgs& p, const float* ubar, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_atom_bwd<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)atom_smem<F>());
        attr = true;
    }
    int grid = (p.n_atoms + AtomTile<F>::A - 1) / AtomTile<F>::A;
    k_atom_bwd<F><<<grid, kAT, atom_smem<F>(), s>>>(p, ubar);
}

}  // namespace

void launch_atom_fwd(const PotArgs& p, int F, const float* msg, cudaStream_t s) {
    if (p.n_atoms == 0) return;
    if (F == 64) atom_fwd_go<64>(p, msg, s);
    else atom_fwd_go<32>(p, msg, s);
    count_launch();
}

void launch_atom_bwd(const PotArgs& p, int F, const float* ubar, cudaStream_t s) {
    if (p.n_atoms == 0) return;
    if (F == 64) atom_bwd_go<64>(p, ubar, s);
    else atom_bwd_go<32>(p, ubar, s);
    count_launch();
}

}  // namespace dmts
