// Per-atom MLPs of the potential (FP32, register-blocked SIMT), run after the
// edge passes have produced the per-atom sums: in the FP32 mode, and in the
// BF16 mode for models narrower than F = 64 (wider ones use the tensor-core
// kernels of atom_tc.cu):
//
//   forward, layer l:   z = m U1 + c1;  h <- h + SiLU(z) U2 + c2;
//                       l < L-1:  u^{l+1} = h W_in^{l+1}
//                       l = L-1:  q = h R1 + d1;  E_i = SiLU(q) . R2 + d2 + e0[Z_i] + E_rep,i
//                                 and the first adjoint steps:
//                                 gh = (SiLU'(q) * R2) R1^T;  mbar^l = ((gh U2^T) * SiLU'(z)) U1^T
//   backward, layer l >= 1:  gh <- gh + ubar^l W_in^{l T};
//                            mbar^{l-1} = ((gh U2^{l-1 T}) * SiLU'(z^{l-1})) U1^{l-1 T}
//
// Layer 0 reads h^0 = A[Z_i] from the per-atom copy built once per parameter
// upload. A CTA takes A = 32 atoms; each stage is an [A x F] x [F x F]
// product, each thread owning RA atoms x RF features (4 x 4 at F = 64; 4 x 2
// at F = 32, so that the narrow model still has 4 warps per CTA). Inputs stay in their
// natural [atom][k] layout in shared memory; the weight matrix of the next
// stage (row-major; the transposed ones are copies prepared on the host)
// streams in with cp.async while the current stage computes.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace dmts {

namespace {

template <int F>
struct AtomTile {
    static constexpr int A = 32;            // atoms per CTA
    static constexpr int RA = 4;            // atoms per thread
    static constexpr int RF = F >= 64 ? 4 : 2;  // features per thread
    static constexpr int FG = F / RF;       // feature groups
    static constexpr int NT = (A / RA) * FG; // threads per CTA: 128
    static constexpr int XS = F + 4;        // row stride of per-atom rows [a][k]
    static constexpr int WS = F + 4;        // row stride of staged weights [k][f]
    static constexpr int SMEM = (2 * A * XS + 2 * F * WS) * 4;
    static_assert(FG <= 32 && 32 % FG == 0, "an atom's feature groups are lanes of one warp");
};

__device__ __forceinline__ float sig(float x) { return 1.0f / (1.0f + __expf(-x)); }

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem))), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// RF consecutive floats (RF = 2 or 4, aligned to RF floats) to and from registers.
template <int RF>
__device__ __forceinline__ void ld_vec(float (&d)[RF], const float* s) {
    if constexpr (RF == 4) {
        const float4 x = *reinterpret_cast<const float4*>(s);
        d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
    } else {
        const float2 x = *reinterpret_cast<const float2*>(s);
        d[0] = x.x; d[1] = x.y;
    }
}
template <int RF>
__device__ __forceinline__ void st_vec(float* d, const float (&v)[RF]) {
    if constexpr (RF == 4) *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<float2*>(d) = make_float2(v[0], v[1]);
}

// Start copying the row-major F x F matrix W into Ws [F][WS] (closes a commit group).
template <int F>
__device__ __forceinline__ void stage_w(float* Ws, const float* __restrict__ W) {
    using T = AtomTile<F>;
    for (int t = threadIdx.x; t < F * F / 4; t += T::NT) {
        const int r = t / (F / 4), c = (t % (F / 4)) * 4;
        cp_async16(Ws + r * T::WS + c, W + (size_t)r * F + c);
    }
    cp_commit();
}

// Start copying rows base .. base + A - 1 of the [N][F] array src into X [A][XS]
// (rows past N are zero); joins the next commit group.
template <int F>
__device__ __forceinline__ void stage_rows(float* X, const float* __restrict__ src, int base, int n_atoms) {
    using T = AtomTile<F>;
    for (int t = threadIdx.x; t < T::A * F / 4; t += T::NT) {
        const int a = t / (F / 4), c = (t % (F / 4)) * 4;
        if (base + a < n_atoms) cp_async16(X + a * T::XS + c, src + (size_t)(base + a) * F + c);
        else *reinterpret_cast<float4*>(X + a * T::XS + c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// acc[a][f] = sum_k X[a0 + a][k] * Ws[k][f0 + f], k ascending.
template <int F>
__device__ __forceinline__ void gemm_blk(const float* X, const float* Ws, int a0, int f0,
                                         float (&acc)[AtomTile<F>::RA][AtomTile<F>::RF]) {
    using T = AtomTile<F>;
#pragma unroll
    for (int a = 0; a < T::RA; ++a)
#pragma unroll
        for (int f = 0; f < T::RF; ++f) acc[a][f] = 0.f;
#pragma unroll 4
    for (int k = 0; k < F; k += 4) {
        float xv[T::RA][4];
#pragma unroll
        for (int a = 0; a < T::RA; ++a) ld_vec<4>(xv[a], X + (a0 + a) * T::XS + k);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            float w[T::RF];
            ld_vec<T::RF>(w, Ws + (k + kk) * T::WS + f0);
#pragma unroll
            for (int a = 0; a < T::RA; ++a)
#pragma unroll
                for (int f = 0; f < T::RF; ++f) acc[a][f] += xv[a][kk] * w[f];
        }
    }
}

template <int F>
__device__ __forceinline__ void put_rows(float* X, int a0, int f0,
                                         const float (&v)[AtomTile<F>::RA][AtomTile<F>::RF]) {
    using T = AtomTile<F>;
#pragma unroll
    for (int a = 0; a < T::RA; ++a) st_vec<T::RF>(X + (a0 + a) * T::XS + f0, v[a]);
}

template <int F>
__device__ __forceinline__ void store_rows(float* __restrict__ dst, int base, int n_atoms, int a0, int f0,
                                           const float (&v)[AtomTile<F>::RA][AtomTile<F>::RF]) {
    using T = AtomTile<F>;
#pragma unroll
    for (int a = 0; a < T::RA; ++a) {
        const int i = base + a0 + a;
        if (i < n_atoms) st_vec<T::RF>(dst + (size_t)i * F + f0, v[a]);
    }
}

// BF16 copy of the same block into interleaved rows (F * 4 bytes per atom;
// per 16 features 16 u values then 16 mbar values, half 0 or 1).
template <int F>
__device__ __forceinline__ void store_rows_bf16(unsigned char* __restrict__ dst, int half, int base, int n_atoms,
                                                int a0, int f0, const float (&v)[AtomTile<F>::RA][AtomTile<F>::RF]) {
    using T = AtomTile<F>;
    if (!dst) return;
#pragma unroll
    for (int a = 0; a < T::RA; ++a) {
        const int i = base + a0 + a;
        if (i >= n_atoms) continue;
        unsigned char* row = dst + (size_t)i * F * 4 + (f0 >> 4) * 64 + half * 32 + (f0 & 15) * 2;
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[a][0], v[a][1]);
        if constexpr (T::RF == 4) {
            __nv_bfloat162 hi = __floats2bfloat162_rn(v[a][2], v[a][3]);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t*>(&lo);
            w.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(row) = w;
        } else {
            *reinterpret_cast<uint32_t*>(row) = *reinterpret_cast<uint32_t*>(&lo);
        }
    }
}

template <int F>
__device__ __forceinline__ void load_rows(float (&v)[AtomTile<F>::RA][AtomTile<F>::RF], const float* __restrict__ src,
                                          int base, int n_atoms, int a0, int f0) {
    using T = AtomTile<F>;
#pragma unroll
    for (int a = 0; a < T::RA; ++a) {
        const int i = base + a0 + a;
        if (i < n_atoms) {
            ld_vec<T::RF>(v[a], src + (size_t)i * F + f0);
        } else {
#pragma unroll
            for (int f = 0; f < T::RF; ++f) v[a][f] = 0.f;
        }
    }
}

// Transposed F x F copies: W_in^T, U1^T, U2^T of every layer, then R1^T.
__device__ __forceinline__ const float* wt_of(const PotArgs& p, int F, int l, int which) {
    return p.PT + ((size_t)3 * l + which) * F * F;
}
__device__ __forceinline__ const float* r1t_of(const PotArgs& p, int F) {
    return p.PT + (size_t)3 * p.n_layers * F * F;
}

template <int F>
__global__ void __launch_bounds__(AtomTile<F>::NT) k_atom_fwd(PotArgs p, const float* __restrict__ msg) {
    using T = AtomTile<F>;
    extern __shared__ float4 smem4[];
    float* X = reinterpret_cast<float*>(smem4);      // [A][XS]
    float* Y = X + T::A * T::XS;                     // [A][XS]
    float* W0 = Y + T::A * T::XS;                    // [F][WS]
    float* W1 = W0 + F * T::WS;                      // [F][WS]
    __shared__ float sE[T::A];
    __shared__ float sBias[4][F];                    // c1, c2 of this layer; d1, R2 (last layer)
    const int l = p.layer;
    const int base = blockIdx.x * T::A;
    const int tid = threadIdx.x, fg = tid % T::FG, ag = tid / T::FG;
    const int f0 = T::RF * fg, a0 = T::RA * ag;
    const float* P = p.P;
    const bool last = (l == p.n_layers - 1);
    float z[T::RA][T::RF], v[T::RA][T::RF], h[T::RA][T::RF];

    stage_rows<F>(X, msg, base, p.n_atoms);
    stage_w<F>(W0, P + p.off.U1[l]);                                     // group: message rows + U1
    stage_w<F>(W1, P + p.off.U2[l]);                                     // group: U2
    load_rows<F>(h, p.h_in, base, p.n_atoms, a0, f0);
    // the small per-layer vectors and the per-atom energy constants, loaded while the copies run
    for (int t = tid; t < F; t += T::NT) {
        sBias[0][t] = __ldg(P + p.off.c1[l] + t);
        sBias[1][t] = __ldg(P + p.off.c2[l] + t);
        if (last) {
            sBias[2][t] = __ldg(P + p.off.d1 + t);
            sBias[3][t] = __ldg(P + p.off.R2 + t);
        }
    }
    // After a tensor-core forward pass that left its split rows to this kernel
    // (fused_fixup): a row split across 128-pair tiles gets the head tile's
    // last carry slot plus the later tiles' first slots, in tile order, and a
    // row without pairs zeros (the order and sums of the separate fix-up pass).
    auto split_row = [&](int i, long long& t0, long long& t1) -> int {   // 0: in one tile, 1: split, 2: empty
        const long long r0 = min((long long)p.row_ptr[i], p.e_cap), r1 = min((long long)p.row_ptr[i + 1], p.e_cap);
        if (r1 <= r0) return 2;
        t0 = r0 >> 7;
        t1 = (r1 - 1) >> 7;
        return t0 == t1 ? 0 : 1;
    };
    double e_const = 0.0;                            // d2 + e0[Z_i] + E_rep,i of atom base + tid
    if (tid < T::A && base + tid < p.n_atoms && p.energy && (last || (p.fused_fixup && l == 0))) {
        const int i = base + tid;
        float erep = 0.f;
        if (l == 0 && p.fused_fixup) {               // E_rep,i is a scalar slot of the layer-0 pass
            long long t0 = 0, t1 = 0;
            const int k = split_row(i, t0, t1);
            if (k == 0) {
                erep = p.erep[i];
            } else if (k == 1) {
                erep = p.carry[(2 * t0 + 1) * (long long)p.carry_w + F];
                for (long long u = t0 + 1; u <= t1; ++u) erep += p.carry[2 * u * (long long)p.carry_w + F];
            }
            p.erep[i] = erep;                        // read again by the last layer of deeper models
        } else {
            erep = p.erep[i];
        }
        if (last) e_const = (double)__ldg(P + p.off.d2) + (double)__ldg(P + p.off.e0 + p.species[i]) + (double)erep;
    }
    cp_wait<1>();
    __syncthreads();
    if (p.fused_fixup) {
#pragma unroll
        for (int a = 0; a < T::RA; ++a) {
            const int i = base + a0 + a;
            if (i >= p.n_atoms) continue;
            long long t0 = 0, t1 = 0;
            const int k = split_row(i, t0, t1);
            if (k == 0) continue;
            float v[T::RF];
#pragma unroll
            for (int f = 0; f < T::RF; ++f) v[f] = 0.f;
            if (k == 1) {
                ld_vec<T::RF>(v, p.carry + (2 * t0 + 1) * (long long)p.carry_w + f0);
                for (long long u = t0 + 1; u <= t1; ++u) {
                    float w[T::RF];
                    ld_vec<T::RF>(w, p.carry + 2 * u * (long long)p.carry_w + f0);
#pragma unroll
                    for (int f = 0; f < T::RF; ++f) v[f] += w[f];
                }
            }
            st_vec<T::RF>(X + (a0 + a) * T::XS + f0, v);
        }
        __syncthreads();
    }
    gemm_blk<F>(X, W0, a0, f0, z);                                       // z = m U1 + c1
#pragma unroll
    for (int f = 0; f < T::RF; ++f) {
        const float c1 = sBias[0][f0 + f];
#pragma unroll
        for (int a = 0; a < T::RA; ++a) {
            z[a][f] += c1;
            v[a][f] = z[a][f] * sig(z[a][f]);
        }
    }
    // a one-layer model read only for its force needs z, h, dE/dh and E_i of no later kernel
    const bool keep = !(p.lean && p.n_layers == 1);
    if (keep) store_rows<F>(p.z, base, p.n_atoms, a0, f0, z);
    put_rows<F>(Y, a0, f0, v);
    __syncthreads();                                                     // W0 read, Y complete
    stage_w<F>(W0, last ? P + p.off.R1 : P + p.off.W_in[l + 1]);
    cp_wait<1>();
    __syncthreads();
    gemm_blk<F>(Y, W1, a0, f0, v);                                       // h += SiLU(z) U2 + c2
#pragma unroll
    for (int f = 0; f < T::RF; ++f) {
        const float c2 = sBias[1][f0 + f];
#pragma unroll
        for (int a = 0; a < T::RA; ++a) h[a][f] += v[a][f] + c2;
    }
    if (keep) store_rows<F>(p.h, base, p.n_atoms, a0, f0, h);
    put_rows<F>(X, a0, f0, h);
    __syncthreads();                                                     // W1 read, X complete
    if (!last) {
        cp_wait<0>();
        __syncthreads();
        gemm_blk<F>(X, W0, a0, f0, v);                                   // u^{l+1} = h W_in^{l+1}
        store_rows<F>(p.u_next, base, p.n_atoms, a0, f0, v);
        store_rows_bf16<F>(p.um_u_out, 0, base, p.n_atoms, a0, f0, v);
        return;
    }
    stage_w<F>(W1, r1t_of(p, F));
    cp_wait<1>();
    __syncthreads();
    gemm_blk<F>(X, W0, a0, f0, v);                                       // q = h R1 + d1
    float e_part[T::RA];
#pragma unroll
    for (int a = 0; a < T::RA; ++a) e_part[a] = 0.f;
#pragma unroll
    for (int f = 0; f < T::RF; ++f) {
        const float d1 = sBias[2][f0 + f], r2 = sBias[3][f0 + f];
#pragma unroll
        for (int a = 0; a < T::RA; ++a) {
            const float q = v[a][f] + d1;
            const float s = sig(q);
            e_part[a] += q * s * r2;
            v[a][f] = s * (1.f + q * (1.f - s)) * r2;                  // dE/dq
        }
    }
    // sum the energy terms over the FG threads of this atom group (consecutive lanes)
#pragma unroll
    for (int a = 0; a < T::RA; ++a)
#pragma unroll
        for (int o = T::FG / 2; o > 0; o >>= 1) e_part[a] += __shfl_xor_sync(0xffffffffu, e_part[a], o);
    if (fg == 0)
#pragma unroll
        for (int a = 0; a < T::RA; ++a) sE[a0 + a] = e_part[a];
    put_rows<F>(Y, a0, f0, v);
    __syncthreads();                                                     // W0 read, Y and sE complete
    stage_w<F>(W0, wt_of(p, F, l, 2));                                   // U2^T
    static_assert(T::NT >= T::A, "one thread per atom of the tile");
    if (keep && tid < T::A && base + tid < p.n_atoms) p.Ei[base + tid] = (double)sE[tid] + e_const;
    cp_wait<1>();
    __syncthreads();
    gemm_blk<F>(Y, W1, a0, f0, v);                                       // gh = gq R1^T
    if (keep) store_rows<F>(p.gh, base, p.n_atoms, a0, f0, v);
    put_rows<F>(X, a0, f0, v);
    __syncthreads();                                                     // W1 read, X complete
    stage_w<F>(W1, wt_of(p, F, l, 1));                                   // U1^T
    cp_wait<1>();
    __syncthreads();
    gemm_blk<F>(X, W0, a0, f0, v);                                       // gy = gh U2^T
#pragma unroll
    for (int a = 0; a < T::RA; ++a)
#pragma unroll
        for (int f = 0; f < T::RF; ++f) {
            const float s = sig(z[a][f]);
            v[a][f] *= s * (1.f + z[a][f] * (1.f - s));
        }
    put_rows<F>(Y, a0, f0, v);
    cp_wait<0>();
    __syncthreads();
    gemm_blk<F>(Y, W1, a0, f0, v);                                       // mbar = gz U1^T
    store_rows<F>(p.mbar_out, base, p.n_atoms, a0, f0, v);
    store_rows_bf16<F>(p.um_mbar_out, 1, base, p.n_atoms, a0, f0, v);
}

template <int F>
__global__ void __launch_bounds__(AtomTile<F>::NT) k_atom_bwd(PotArgs p, const float* __restrict__ ubar) {
    using T = AtomTile<F>;
    extern __shared__ float4 smem4[];
    float* X = reinterpret_cast<float*>(smem4);
    float* Y = X + T::A * T::XS;
    float* W0 = Y + T::A * T::XS;
    float* W1 = W0 + F * T::WS;
    const int l = p.layer;   // >= 1
    const int base = blockIdx.x * T::A;
    const int tid = threadIdx.x, fg = tid % T::FG, ag = tid / T::FG;
    const int f0 = T::RF * fg, a0 = T::RA * ag;
    float v[T::RA][T::RF], g[T::RA][T::RF], z[T::RA][T::RF];
    stage_rows<F>(X, ubar, base, p.n_atoms);
    stage_w<F>(W0, wt_of(p, F, l, 0));                                   // group: ubar rows + W_in^{l T}
    stage_w<F>(W1, wt_of(p, F, l - 1, 2));                               // group: U2^{l-1 T}
    load_rows<F>(g, p.gh, base, p.n_atoms, a0, f0);
    load_rows<F>(z, p.z_prev, base, p.n_atoms, a0, f0);
    cp_wait<1>();
    __syncthreads();
    gemm_blk<F>(X, W0, a0, f0, v);                                       // ubar W_in^T
#pragma unroll
    for (int a = 0; a < T::RA; ++a)
#pragma unroll
        for (int f = 0; f < T::RF; ++f) g[a][f] += v[a][f];
    store_rows<F>(p.gh, base, p.n_atoms, a0, f0, g);
    put_rows<F>(Y, a0, f0, g);
    __syncthreads();                                                     // W0 read, Y complete
    stage_w<F>(W0, wt_of(p, F, l - 1, 1));                               // U1^{l-1 T}
    cp_wait<1>();
    __syncthreads();
    gemm_blk<F>(Y, W1, a0, f0, v);                                       // gy = gh U2^T
#pragma unroll
    for (int a = 0; a < T::RA; ++a)
#pragma unroll
        for (int f = 0; f < T::RF; ++f) {
            const float s = sig(z[a][f]);
            v[a][f] *= s * (1.f + z[a][f] * (1.f - s));
        }
    put_rows<F>(X, a0, f0, v);
    cp_wait<0>();
    __syncthreads();
    gemm_blk<F>(X, W0, a0, f0, v);                                       // mbar^{l-1} = gz U1^T
    store_rows<F>(p.mbar_out, base, p.n_atoms, a0, f0, v);
    store_rows_bf16<F>(p.um_mbar_out, 1, base, p.n_atoms, a0, f0, v);
}

template <int F>
void atom_fwd_go(const PotArgs& p, const float* msg, cudaStream_t s) {
    using T = AtomTile<F>;
    smem_opt_in((const void*)k_atom_fwd<F>, T::SMEM);
    k_atom_fwd<F><<<(p.n_atoms + T::A - 1) / T::A, T::NT, T::SMEM, s>>>(p, msg);
}

template <int F>
void atom_bwd_go(const PotArgs& p, const float* ubar, cudaStream_t s) {
    using T = AtomTile<F>;
    smem_opt_in((const void*)k_atom_bwd<F>, T::SMEM);
    k_atom_bwd<F><<<(p.n_atoms + T::A - 1) / T::A, T::NT, T::SMEM, s>>>(p, ubar);
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
