// FP32 SIMT path of the potential: forward message passing and the force
// adjoint, with the per-edge filter MLP recomputed (never stored).
//
// Work decomposition: CTA b owns the atoms [b*A, (b+1)*A) and therefore the
// contiguous CSR edge range of their rows. It walks that range in tiles of
// TE edges; within a tile the filter MLP is a register-blocked GEMM (each of
// the 256 threads owns 4 edges x 4 features), and the per-row sums are taken
// in edge order by one thread per feature, so results are deterministic and
// atomic-free. The per-atom sums (messages, or the adjoint ubar) are written
// to global memory for the per-atom MLP kernels.
//
// Adjoint (F = -dE/dx): with g_ij = mbar_i * u_j + mbar_j * u_i (the filter
// depends on d only, so w_ij = w_ji), dE/dd_ij = fc' (g . phi) +
// fc sum_k [(g W2^T)_k SiLU'(a_k)] (e' W1)_k, and F_i = sum_j dE/dd_ij rhat_ij
// over row i; the adjoint of u is ubar_i = sum_j w_ij * mbar_j, again a sum
// over row i. Both are gathers over the atom's own row.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace dmts {

namespace {

template <int K>
__device__ __forceinline__ void basis_fwd(float d, float pi_over_rc, float pref, float* e, float& fc) {
    float s1, c1;
    sincospif(d * (pi_over_rc * 0.31830988618379067f), &s1, &c1);
    float inv_d = 1.0f / d;
    float sk = s1, skm1 = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        e[k] = pref * sk * inv_d;
        float sn = 2.f * c1 * sk - skm1;
        skm1 = sk;
        sk = sn;
    }
    fc = 0.5f * (c1 + 1.0f);
}

template <int K>
__device__ __forceinline__ void basis_bwd(float d, float pi_over_rc, float pref, float* e, float* de,
                                          float& fc, float& dfc) {
    float s1, c1;
    sincospif(d * (pi_over_rc * 0.31830988618379067f), &s1, &c1);
    float inv_d = 1.0f / d;
    float sk = s1, skm1 = 0.f, ck = c1, ckm1 = 1.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float kw = (float)(k + 1) * pi_over_rc;
        e[k] = pref * sk * inv_d;
        de[k] = pref * (kw * ck - sk * inv_d) * inv_d;
        float sn = 2.f * c1 * sk - skm1;
        float cn = 2.f * c1 * ck - ckm1;
        skm1 = sk; sk = sn;
        ckm1 = ck; ck = cn;
    }
    fc = 0.5f * (c1 + 1.0f);
    dfc = -0.5f * pi_over_rc * s1;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float f4(const float4& v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// ------------------------------------------------------------ shared layout
template <int F, int K>
struct Tile {
    static constexpr int TE = 4096 / F;          // edges per tile (EPT = 4)
    static constexpr int FG = F / 4;             // feature groups
    static constexpr int EG = kThreads / FG;     // edge groups
    static constexpr int PS = F + 4;             // row stride of the message tile
    static_assert(EG * 4 == TE, "tile shape");
};

template <int F, int K>
constexpr int fwd_smem_floats(int A) {
    using T = Tile<F, K>;
    return K * F + F + F * F + F + K * T::TE + F * T::TE + T::TE * T::PS + 4 * T::TE + A * F;
}

template <int F, int K>
constexpr int bwd_smem_floats(int A) {
    using T = Tile<F, K>;
    return K * F + F + F * F + F + F * F        // W1 b1 W2 b2 W2T
           + 2 * K * T::TE                      // BT DT
           + 2 * F * T::TE                      // ST GT
           + T::TE * T::PS                      // P
           + 10 * T::TE                         // fc dfc se rh(4) j row pad
           + 2 * T::TE * T::FG                  // red1 red2
           + A * F + A * 4 + A * 8;             // acc force virial
}

// ------------------------------------------------------------ embedding
template <int F>
__global__ void k_embed(PotArgs a) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int i = t / F, f = t % F;
    if (i >= a.n_atoms) return;
    int z = a.species[i];
    const float* A = a.P + a.off.A + z * F;
    const float* W = a.P + a.off.W_in[0];
    float acc = 0.f;
    for (int k = 0; k < F; ++k) acc += __ldg(A + k) * __ldg(W + k * F + f);
    a.h[(size_t)i * F + f] = __ldg(A + f);
    a.u_next[(size_t)i * F + f] = acc;
    if (a.um_u_out)
        *reinterpret_cast<__nv_bfloat16*>(a.um_u_out + (size_t)i * F * 4 + (f >> 4) * 64 + (f & 15) * 2) =
            __float2bfloat16_rn(acc);
}

// ------------------------------------------------------------ forward edge pass
template <int F, int K>
__global__ void __launch_bounds__(kThreads) k_edge_fwd(PotArgs a) {
    using T = Tile<F, K>;
    constexpr int TE = T::TE, FG = T::FG, PS = T::PS;
    extern __shared__ float4 smem4[];
    float* sW1 = reinterpret_cast<float*>(smem4);
    float* sb1 = sW1 + K * F;
    float* sW2 = sb1 + F;
    float* sb2 = sW2 + F * F;
    float* sBT = sb2 + F;
    float* sST = sBT + K * TE;
    float* sP = sST + F * TE;
    float* sfc = sP + TE * PS;
    int* sj = reinterpret_cast<int*>(sfc + TE);
    int* srow = sj + TE;
    float* srep = reinterpret_cast<float*>(srow + TE);
    float* sAcc = srep + TE;
    const int A = a.atoms_per_cta;
    const int tid = threadIdx.x;
    const int l = a.layer;
    const int a0 = blockIdx.x * A;
    const int a1 = min(a.n_atoms, a0 + A);
    const int nA = a1 - a0;
    if (nA <= 0) return;

    for (int t = tid; t < K * F; t += kThreads) sW1[t] = __ldg(a.P + a.off.W1[l] + t);
    for (int t = tid; t < F * F; t += kThreads) sW2[t] = __ldg(a.P + a.off.W2[l] + t);
    for (int t = tid; t < F; t += kThreads) {
        sb1[t] = __ldg(a.P + a.off.b1[l] + t);
        sb2[t] = __ldg(a.P + a.off.b2[l] + t);
    }
    for (int t = tid; t < A * F; t += kThreads) sAcc[t] = 0.f;
    // layer 0 also sums the pair repulsion, 1/2 phi(d_ij) per directed pair
    if (l == 0)
        for (int t = tid; t < nA; t += kThreads) a.erep[a0 + t] = 0.f;

    const long long e_beg = min((long long)a.row_ptr[a0], a.e_cap);
    const long long e_end = min((long long)a.row_ptr[a1], a.e_cap);
    const int fg = tid % FG, eg = tid / FG;
    const int f0 = fg * 4, e0 = eg * 4;
    int cur = -1;
    float run = 0.f;
    __syncthreads();

    for (long long t0 = e_beg; t0 < e_end; t0 += TE) {
        if (tid < TE) {
            long long e = t0 + tid;
            float eb[K];
            if (e < e_end) {
                int j = DMTS_IDX(a.col[e], a.n_atoms, a.check), i = DMTS_IDX(a.recv[e], a.n_atoms, a.check);
                uint4 qi = a.q[i], qj = a.q[j];
                float3 r = edge_vec(qi, qj, a.frame[qi.w].qscale);
                float d = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
                float fc;
                basis_fwd<K>(d, a.pi_over_rc, a.bessel_pref, eb, fc);
                sfc[tid] = fc;
                sj[tid] = j;
                srow[tid] = i - a0;
                srep[tid] = l == 0 ? 0.5f * rep_phi(d, a.rep_a, a.rep_inv_rho, a.rep_rc, a.rep_pi_over_rc, nullptr) : 0.f;
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) eb[k] = 0.f;
                sfc[tid] = 0.f;
                sj[tid] = a0;
                srow[tid] = -1;
                srep[tid] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < K; ++k) sBT[k * TE + tid] = eb[k];
        }
        __syncthreads();
        // GEMM 1: hidden = SiLU(e W1 + b1), stored transposed
        {
            float acc[4][4];
            float4 b = ld4(sb1 + f0);
#pragma unroll
            for (int r = 0; r < 4; ++r) { acc[r][0] = b.x; acc[r][1] = b.y; acc[r][2] = b.z; acc[r][3] = b.w; }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float4 bv = ld4(sBT + k * TE + e0);
                float4 wv = ld4(sW1 + k * F + f0);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += f4(bv, r) * f4(wv, c);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float sg, s[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) s[r] = silu_f(acc[r][c], sg);
                st4(sST + (f0 + c) * TE + e0, make_float4(s[0], s[1], s[2], s[3]));
            }
        }
        __syncthreads();
        // GEMM 2: phi = hidden W2 + b2; message = fc * phi * u_j
        {
            float acc[4][4];
            float4 b = ld4(sb2 + f0);
#pragma unroll
            for (int r = 0; r < 4; ++r) { acc[r][0] = b.x; acc[r][1] = b.y; acc[r][2] = b.z; acc[r][3] = b.w; }
#pragma unroll 4
            for (int k = 0; k < F; ++k) {
                float4 sv = ld4(sST + k * TE + e0);
                float4 wv = ld4(sW2 + k * F + f0);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += f4(sv, r) * f4(wv, c);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int e = e0 + r;
                float fc = sfc[e];
                float4 uj = ldg4(a.u + (size_t)sj[e] * F + f0);
                st4(sP + e * PS + f0, make_float4(fc * acc[r][0] * uj.x, fc * acc[r][1] * uj.y,
                                                  fc * acc[r][2] * uj.z, fc * acc[r][3] * uj.w));
            }
        }
        __syncthreads();
        // segmented row sums, in edge order (thread F: repulsion energy)
        if (tid < F) {
            for (int e = 0; e < TE; ++e) {
                int r = srow[e];
                if (r < 0) break;
                if (r != cur) {
                    if (cur >= 0) sAcc[cur * F + tid] = run;
                    cur = r;
                    run = 0.f;
                }
                run += sP[e * PS + tid];
            }
        } else if (tid == F && l == 0) {
            for (int e = 0; e < TE; ++e) {
                int r = srow[e];
                if (r < 0) break;
                if (r != cur) {
                    if (cur >= 0) a.erep[a0 + cur] = run;
                    cur = r;
                    run = 0.f;
                }
                run += srep[e];
            }
        }
        __syncthreads();
    }
    if (tid < F && cur >= 0) sAcc[cur * F + tid] = run;
    if (tid == F && l == 0 && cur >= 0) a.erep[a0 + cur] = run;

    __syncthreads();
    for (int t = tid; t < nA * F; t += kThreads) a.msg_out[(size_t)a0 * F + t] = sAcc[t];
}

// ------------------------------------------------------------ backward edge pass
template <int F, int K>
__global__ void __launch_bounds__(kThreads) k_edge_bwd(PotArgs a) {
    using T = Tile<F, K>;
    constexpr int TE = T::TE, FG = T::FG, PS = T::PS;
    extern __shared__ float4 smem4[];
    float* sW1 = reinterpret_cast<float*>(smem4);
    float* sb1 = sW1 + K * F;
    float* sW2 = sb1 + F;
    float* sb2 = sW2 + F * F;
    float* sW2T = sb2 + F;
    float* sBT = sW2T + F * F;
    float* sDT = sBT + K * TE;
    float* sST = sDT + K * TE;
    float* sGT = sST + F * TE;
    float* sP = sGT + F * TE;
    float* sfc = sP + TE * PS;
    float* sdfc = sfc + TE;
    float* sse = sdfc + TE;
    float* srh = sse + TE;                       // [TE][4] rhat, d
    int* sj = reinterpret_cast<int*>(srh + 4 * TE);
    int* srow = sj + TE;
    float* red1 = reinterpret_cast<float*>(srow + TE) + TE;  // one pad block
    float* red2 = red1 + TE * FG;
    float* sAcc = red2 + TE * FG;                // [A][F] ubar
    float* sF = sAcc + a.atoms_per_cta * F;      // [A][4]
    float* sV = sF + a.atoms_per_cta * 4;        // [A][8]
    const int A = a.atoms_per_cta;
    const int tid = threadIdx.x;
    const int l = a.layer;
    const int a0 = blockIdx.x * A;
    const int a1 = min(a.n_atoms, a0 + A);
    const int nA = a1 - a0;
    if (nA <= 0) return;
    const bool need_ubar = (l > 0);

    for (int t = tid; t < K * F; t += kThreads) sW1[t] = __ldg(a.P + a.off.W1[l] + t);
    for (int t = tid; t < F * F; t += kThreads) {
        float w = __ldg(a.P + a.off.W2[l] + t);
        sW2[t] = w;
        sW2T[(t % F) * F + t / F] = w;
    }
    for (int t = tid; t < F; t += kThreads) {
        sb1[t] = __ldg(a.P + a.off.b1[l] + t);
        sb2[t] = __ldg(a.P + a.off.b2[l] + t);
    }
    for (int t = tid; t < A * F; t += kThreads) sAcc[t] = 0.f;
    for (int t = tid; t < A * 12; t += kThreads) sF[t] = 0.f;   // sF and sV are adjacent

    const long long e_beg = min((long long)a.row_ptr[a0], a.e_cap);
    const long long e_end = min((long long)a.row_ptr[a1], a.e_cap);
    const int fg = tid % FG, eg = tid / FG;
    const int f0 = fg * 4, e0 = eg * 4;
    // running sums: threads [128, 128+F) for ubar, threads [0, 9) for force/virial
    int cur = -1;
    float run = 0.f;
    __syncthreads();

    for (long long t0 = e_beg; t0 < e_end; t0 += TE) {
        if (tid < TE) {
            long long e = t0 + tid;
            float eb[K], db[K];
            if (e < e_end) {
                int j = DMTS_IDX(a.col[e], a.n_atoms, a.check), i = DMTS_IDX(a.recv[e], a.n_atoms, a.check);
                uint4 qi = a.q[i], qj = a.q[j];
                float3 r = edge_vec(qi, qj, a.frame[qi.w].qscale);
                float d = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
                float fc, dfc;
                basis_bwd<K>(d, a.pi_over_rc, a.bessel_pref, eb, db, fc, dfc);
                float inv = 1.0f / d;
                sfc[tid] = fc;
                sdfc[tid] = dfc;
                st4(srh + 4 * tid, make_float4(r.x * inv, r.y * inv, r.z * inv, d));
                sj[tid] = j;
                srow[tid] = i - a0;
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) { eb[k] = 0.f; db[k] = 0.f; }
                sfc[tid] = 0.f;
                sdfc[tid] = 0.f;
                st4(srh + 4 * tid, make_float4(0.f, 0.f, 0.f, 0.f));
                sj[tid] = a0;
                srow[tid] = -1;
            }
#pragma unroll
            for (int k = 0; k < K; ++k) { sBT[k * TE + tid] = eb[k]; sDT[k * TE + tid] = db[k]; }
        }
        __syncthreads();
        // GEMM 1 (+ its derivative companion): a = e W1 + b1, T = e' W1
        float sp[4][4], tt[4][4];
        {
            float acc[4][4];
            float4 b = ld4(sb1 + f0);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                acc[r][0] = b.x; acc[r][1] = b.y; acc[r][2] = b.z; acc[r][3] = b.w;
#pragma unroll
                for (int c = 0; c < 4; ++c) tt[r][c] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float4 bv = ld4(sBT + k * TE + e0);
                float4 dv = ld4(sDT + k * TE + e0);
                float4 wv = ld4(sW1 + k * F + f0);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[r][c] += f4(bv, r) * f4(wv, c);
                        tt[r][c] += f4(dv, r) * f4(wv, c);
                    }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float s[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float sg;
                    s[r] = silu_f(acc[r][c], sg);
                    sp[r][c] = sg * (1.f + acc[r][c] * (1.f - sg));
                }
                st4(sST + (f0 + c) * TE + e0, make_float4(s[0], s[1], s[2], s[3]));
            }
        }
        __syncthreads();
        // GEMM 2: phi = s W2 + b2; g = mbar_i u_j + mbar_j u_i; partial g.phi;
        // G^T for GEMM 3; ubar message w * mbar_j
        {
            float acc[4][4];
            float4 b = ld4(sb2 + f0);
#pragma unroll
            for (int r = 0; r < 4; ++r) { acc[r][0] = b.x; acc[r][1] = b.y; acc[r][2] = b.z; acc[r][3] = b.w; }
#pragma unroll 4
            for (int k = 0; k < F; ++k) {
                float4 sv = ld4(sST + k * TE + e0);
                float4 wv = ld4(sW2 + k * F + f0);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += f4(sv, r) * f4(wv, c);
            }
            float g[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int e = e0 + r;
                int j = sj[e];
                int rr = srow[e];
                int i = rr < 0 ? a0 : a0 + rr;
                float4 uj = ldg4(a.u + (size_t)j * F + f0);
                float4 mj = ldg4(a.mbar + (size_t)j * F + f0);
                float4 ui = ldg4(a.u + (size_t)i * F + f0);
                float4 mi = ldg4(a.mbar + (size_t)i * F + f0);
                g[r][0] = mi.x * uj.x + mj.x * ui.x;
                g[r][1] = mi.y * uj.y + mj.y * ui.y;
                g[r][2] = mi.z * uj.z + mj.z * ui.z;
                g[r][3] = mi.w * uj.w + mj.w * ui.w;
                float dot = g[r][0] * acc[r][0] + g[r][1] * acc[r][1] + g[r][2] * acc[r][2] + g[r][3] * acc[r][3];
                red1[e * FG + fg] = dot;
                if (need_ubar) {
                    float fc = sfc[e];
                    st4(sP + e * PS + f0, make_float4(fc * acc[r][0] * mj.x, fc * acc[r][1] * mj.y,
                                                      fc * acc[r][2] * mj.z, fc * acc[r][3] * mj.w));
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                st4(sGT + (f0 + c) * TE + e0, make_float4(g[0][c], g[1][c], g[2][c], g[3][c]));
        }
        __syncthreads();
        // GEMM 3: abar = G W2^T; partial sum_k abar_k SiLU'(a_k) T_k
        {
            float acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 4
            for (int k = 0; k < F; ++k) {
                float4 gv = ld4(sGT + k * TE + e0);
                float4 wv = ld4(sW2T + k * F + f0);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += f4(gv, r) * f4(wv, c);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float p = 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) p += acc[r][c] * sp[r][c] * tt[r][c];
                red2[(e0 + r) * FG + fg] = p;
            }
        }
        __syncthreads();
        // per-edge dE/dd, and the ubar row sums (threads 128..128+F)
        if (tid < TE) {
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int k = 0; k < FG; ++k) { s1 += red1[tid * FG + k]; s2 += red2[tid * FG + k]; }
            float se = sdfc[tid] * s1 + sfc[tid] * s2;
            if (l == 0 && srow[tid] >= 0) {
                float dphi;
                (void)rep_phi(srh[4 * tid + 3], a.rep_a, a.rep_inv_rho, a.rep_rc, a.rep_pi_over_rc, &dphi);
                se += dphi;
            }
            sse[tid] = se;
        } else if (need_ubar && tid >= 128 && tid < 128 + F) {
            int ff = tid - 128;
            for (int e = 0; e < TE; ++e) {
                int r = srow[e];
                if (r < 0) break;
                if (r != cur) {
                    if (cur >= 0) sAcc[cur * F + ff] = run;
                    cur = r;
                    run = 0.f;
                }
                run += sP[e * PS + ff];
            }
        }
        __syncthreads();
        // force (3) and virial (6) row sums, in edge order
        if (tid < 9) {
            for (int e = 0; e < TE; ++e) {
                int r = srow[e];
                if (r < 0) break;
                if (r != cur) {
                    if (cur >= 0) {
                        if (tid < 3) sF[cur * 4 + tid] = run;
                        else sV[cur * 8 + tid - 3] = run;
                    }
                    cur = r;
                    run = 0.f;
                }
                float4 rh = ld4(srh + 4 * e);
                float s = sse[e];
                float val;
                if (tid < 3) {
                    val = s * f4(rh, tid);
                } else {
                    // W_ab = -1/2 sum_directed s d rhat_a rhat_b; components xx yy zz xy xz yz
                    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
                    int c = tid - 3;
                    val = -0.5f * s * rh.w * f4(rh, ia[c]) * f4(rh, ib[c]);
                }
                run += val;
            }
        }
        __syncthreads();
    }
    if (cur >= 0) {
        if (tid < 3) sF[cur * 4 + tid] = run;
        else if (tid < 9) sV[cur * 8 + tid - 3] = run;
        else if (tid >= 128 && tid < 128 + F) sAcc[cur * F + tid - 128] = run;
    }
    __syncthreads();
    // forces / virial of the CTA's atoms
    for (int t = tid; t < nA * 3; t += kThreads) {
        int r = t / 3, c = t % 3;
        size_t o = (size_t)c * a.n_atoms + a0 + r;
        a.force[o] = a.accumulate ? a.force[o] + sF[r * 4 + c] : sF[r * 4 + c];
    }
    for (int t = tid; t < nA * 6; t += kThreads) {
        int r = t / 6, c = t % 6;
        size_t o = (size_t)(a0 + r) * 6 + c;
        a.vir6[o] = a.accumulate ? a.vir6[o] + sV[r * 8 + c] : sV[r * 8 + c];
    }
    if (need_ubar)
        for (int t = tid; t < nA * F; t += kThreads) a.msg_out[(size_t)a0 * F + t] = sAcc[t];
}

template <int F, int K>
void set_smem_attrs() {
    smem_opt_in((const void*)k_edge_fwd<F, K>, 227 * 1024);
    smem_opt_in((const void*)k_edge_bwd<F, K>, 227 * 1024);
}

template <int F, int K>
void fwd_launch(const PotArgs& a, cudaStream_t s) {
    set_smem_attrs<F, K>();
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    size_t smem = sizeof(float) * fwd_smem_floats<F, K>(a.atoms_per_cta);
    k_edge_fwd<F, K><<<grid, kThreads, smem, s>>>(a);
}

template <int F, int K>
void bwd_launch(const PotArgs& a, cudaStream_t s) {
    set_smem_attrs<F, K>();
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    size_t smem = sizeof(float) * bwd_smem_floats<F, K>(a.atoms_per_cta);
    k_edge_bwd<F, K><<<grid, kThreads, smem, s>>>(a);
}

template <int F>
int max_atoms(int K, bool bwd) {
    // largest A whose shared memory fits
    int best = 0;
    for (int A = 8; A <= 256; A += 8) {
        long long fl;
        long long region;
        switch (K) {
            default: return 0;
#define DMTS_K(KK)                                                                   \
    case KK:                                                                         \
        fl = bwd ? bwd_smem_floats<F, KK>(A) : fwd_smem_floats<F, KK>(A);            \
        break;
            DMTS_K(1) DMTS_K(2) DMTS_K(3) DMTS_K(4) DMTS_K(5) DMTS_K(6) DMTS_K(7) DMTS_K(8)
            DMTS_K(9) DMTS_K(10) DMTS_K(11) DMTS_K(12) DMTS_K(13) DMTS_K(14) DMTS_K(15) DMTS_K(16)
#undef DMTS_K
        }
        (void)region;
        region = 0;
        if (fl * 4 <= 227 * 1024) best = A;
    }
    return best;
}

}  // namespace

#define DMTS_DISPATCH(FN, F_, K_, ...)                                                       \
    do {                                                                                     \
        bool ok_ = false;                                                                    \
        if (F_ == 64) {                                                                      \
            switch (K_) {                                                                    \
                case 1: FN<64, 1>(__VA_ARGS__); ok_ = true; break;                           \
                case 2: FN<64, 2>(__VA_ARGS__); ok_ = true; break;                           \
                case 3: FN<64, 3>(__VA_ARGS__); ok_ = true; break;                           \
                case 4: FN<64, 4>(__VA_ARGS__); ok_ = true; break;                           \
                case 5: FN<64, 5>(__VA_ARGS__); ok_ = true; break;                           \
                case 6: FN<64, 6>(__VA_ARGS__); ok_ = true; break;                           \
                case 7: FN<64, 7>(__VA_ARGS__); ok_ = true; break;                           \
                case 8: FN<64, 8>(__VA_ARGS__); ok_ = true; break;                           \
                case 9: FN<64, 9>(__VA_ARGS__); ok_ = true; break;                           \
                case 10: FN<64, 10>(__VA_ARGS__); ok_ = true; break;                         \
                case 11: FN<64, 11>(__VA_ARGS__); ok_ = true; break;                         \
                case 12: FN<64, 12>(__VA_ARGS__); ok_ = true; break;                         \
                case 13: FN<64, 13>(__VA_ARGS__); ok_ = true; break;                         \
                case 14: FN<64, 14>(__VA_ARGS__); ok_ = true; break;                         \
                case 15: FN<64, 15>(__VA_ARGS__); ok_ = true; break;                         \
                case 16: FN<64, 16>(__VA_ARGS__); ok_ = true; break;                         \
            }                                                                                \
        } else if (F_ == 32) {                                                               \
            switch (K_) {                                                                    \
                case 1: FN<32, 1>(__VA_ARGS__); ok_ = true; break;                           \
                case 2: FN<32, 2>(__VA_ARGS__); ok_ = true; break;                           \
                case 3: FN<32, 3>(__VA_ARGS__); ok_ = true; break;                           \
                case 4: FN<32, 4>(__VA_ARGS__); ok_ = true; break;                           \
                case 5: FN<32, 5>(__VA_ARGS__); ok_ = true; break;                           \
                case 6: FN<32, 6>(__VA_ARGS__); ok_ = true; break;                           \
                case 7: FN<32, 7>(__VA_ARGS__); ok_ = true; break;                           \
                case 8: FN<32, 8>(__VA_ARGS__); ok_ = true; break;                           \
                case 9: FN<32, 9>(__VA_ARGS__); ok_ = true; break;                           \
                case 10: FN<32, 10>(__VA_ARGS__); ok_ = true; break;                         \
                case 11: FN<32, 11>(__VA_ARGS__); ok_ = true; break;                         \
                case 12: FN<32, 12>(__VA_ARGS__); ok_ = true; break;                         \
                case 13: FN<32, 13>(__VA_ARGS__); ok_ = true; break;                         \
                case 14: FN<32, 14>(__VA_ARGS__); ok_ = true; break;                         \
                case 15: FN<32, 15>(__VA_ARGS__); ok_ = true; break;                         \
                case 16: FN<32, 16>(__VA_ARGS__); ok_ = true; break;                         \
            }                                                                                \
        }                                                                                    \
        (void)sizeof(ok_);                                                                   \
    } while (0)

void launch_embed(const PotArgs& a, int F, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    int total = a.n_atoms * F;
    if (F == 64) k_embed<64><<<(total + 255) / 256, 256, 0, s>>>(a);
    else k_embed<32><<<(total + 255) / 256, 256, 0, s>>>(a);
    count_launch();
}

void launch_edge_fwd_f32(const PotArgs& a, int F, int K, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    DMTS_DISPATCH(fwd_launch, F, K, a, s);
    count_launch();
}

void launch_edge_bwd_f32(const PotArgs& a, int F, int K, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    DMTS_DISPATCH(bwd_launch, F, K, a, s);
    count_launch();
}

int max_atoms_per_cta_f32(int F, int K, bool bwd) {
    if (F == 64) return max_atoms<64>(K, bwd);
    if (F == 32) return max_atoms<32>(K, bwd);
    return 0;
}

// ------------------------------------------------------------ reductions
// Per-system FP64 sums in a fixed order (deterministic): one CTA per system,
// strided partial sums, then fixed-shape shuffle trees (deterministic).
template <int NT>
__global__ void __launch_bounds__(NT) k_system_sum(int n_sys, const int* __restrict__ off,
                                                  const double* __restrict__ v, double* __restrict__ out,
                                                  int stride) {
    __shared__ double wsum[NT / 32];
    const int s = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double acc = 0.0;
    for (int i = off[s] + threadIdx.x; i < off[s + 1]; i += NT) acc += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[w] = acc;
    __syncthreads();
    if (w == 0) {
        double t = lane < NT / 32 ? wsum[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) out[(size_t)s * stride] = t;
    }
}

// A few large systems: each system's values in kSumChunks consecutive
// chunks, one CTA per chunk (fixed-order partial sums); the CTA of a system
// that finishes last adds the partials in chunk order and clears the
// system's counter. The FP64 additions spread over many SMs.
template <int NT>
__global__ void __launch_bounds__(NT) k_system_sum_split(const int* __restrict__ off, const double* __restrict__ v,
                                                        double* __restrict__ out, int stride,
                                                        double* __restrict__ part, unsigned int* __restrict__ ctr) {
    __shared__ double wsum[NT / 32];
    __shared__ bool last;
    const int s = blockIdx.y, b = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int begin = off[s], end = off[s + 1];
    const int per = (end - begin + kSumChunks - 1) / kSumChunks;
    const int lo = begin + b * per, hi = min(end, lo + per);
    double acc = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += NT) acc += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < NT / 32; ++k) t += wsum[k];
        part[(size_t)s * kSumChunks + b] = t;
        __threadfence();
        last = atomicAdd(&ctr[s], 1u) == (unsigned int)kSumChunks - 1u;
    }
    __syncthreads();
    if (last && w == 0) {
        __threadfence();
        double u = 0.0;
        for (int k = lane; k < kSumChunks; k += 32) u += __ldcg(part + (size_t)s * kSumChunks + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
        if (lane == 0) {
            out[(size_t)s * stride] = u;
            ctr[s] = 0u;
        }
    }
}

void launch_system_sum(int n_sys, const int* atom_offset, const double* per_atom, double* out,
                       int stride, const SumScratch& sc, cudaStream_t s) {
    if (n_sys <= kSumMaxSplit && sc.part) {
        k_system_sum_split<256><<<dim3(kSumChunks, n_sys), 256, 0, s>>>(atom_offset, per_atom, out, stride, sc.part,
                                                                         sc.ctr);
    } else if (n_sys <= 8) {
        // one CTA per system: wide for a single large system, narrow for many molecules
        k_system_sum<1024><<<n_sys, 1024, 0, s>>>(n_sys, atom_offset, per_atom, out, stride);
    } else {
        k_system_sum<64><<<n_sys, 64, 0, s>>>(n_sys, atom_offset, per_atom, out, stride);
    }
    count_launch();
}

__global__ void k_virial_sum(int n_sys, const int* __restrict__ off, const float* __restrict__ v6,
                             double* __restrict__ out) {
    __shared__ double sh[6][128];
    int s = blockIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x)
        for (int c = 0; c < 6; ++c) acc[c] += (double)v6[(size_t)i * 6 + c];
    for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = out + (size_t)s * 9;
        o[0] = sh[0][0]; o[4] = sh[1][0]; o[8] = sh[2][0];
        o[1] = o[3] = sh[3][0];
        o[2] = o[6] = sh[4][0];
        o[5] = o[7] = sh[5][0];
    }
}

void launch_virial_sum(int n_sys, const int* atom_offset, const float* vir6, double* out,
                       cudaStream_t s) {
    k_virial_sum<<<n_sys, 128, 0, s>>>(n_sys, atom_offset, vir6, out);
    count_launch();
}

}  // namespace dmts
