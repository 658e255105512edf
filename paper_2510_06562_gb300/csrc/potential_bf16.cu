// BF16 tensor-core path of the potential (DMTS_BF16_MLP): the per-edge filter
// MLP runs on the 5th-generation tensor cores (tcgen05.mma, BF16 operands in
// shared memory, FP32 accumulators in tensor memory); edge geometry, message
// sums, forces and the per-atom MLPs stay FP32.
//
// A CTA of 4 warps owns a contiguous range of atoms (whole CSR rows) and walks
// its edges in tiles of 128: one edge per thread and per TMEM lane, so after
// each MMA a thread loads its own edge's full feature row from TMEM.
//   forward, per tile:  A1 = basis (128 x 16)           D1 = A1 W1        (hidden pre-activation)
//                       A2 = SiLU(D1 + b1) (128 x F)    D2 = A2 W2        (filter, w = fc (D2 + b2))
//   backward, per tile: D1 = A1 W1, D4 = A1' W1 (basis derivative), D2 = SiLU(D1 + b1) W2,
//                       g = mbar_i u_j + mbar_j u_i,  D3 = g W2^T,
//                       dE/dd = fc' (g . (D2 + b2)) + fc sum_k D3_k SiLU'(D1_k + b1_k) D4_k.
// The MMAs are issued by one thread; completion is signalled through an
// mbarrier (bounded waits: a wait that gives up sets the timeout flag and the
// kernel finishes without further MMAs, freeing its tensor memory).
#include "internal.cuh"
#include "umma.cuh"

namespace dmts {

namespace {

using namespace umma;

constexpr int kT = 128;          // threads per CTA = edges per tile = TMEM lanes
constexpr int kKP = 16;          // radial functions padded to one MMA K step
constexpr uint32_t kWaitIter = 1u << 22;

__device__ __forceinline__ float sigmoid_fast(float x) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * x));
    return fmaf(0.5f, t, 0.5f);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Store 8 consecutive K values (k0 multiple of 8) of row r as bf16.
__device__ __forceinline__ void st_row8(unsigned char* tile, int r, int k0, int Kc, const float* v) {
    uint4 q;
    q.x = pack_bf16(v[0], v[1]);
    q.y = pack_bf16(v[2], v[3]);
    q.z = pack_bf16(v[4], v[5]);
    q.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + tile_offset(r, k0, Kc)) = q;
}

// Bessel basis (K <= 16 functions, padded with zeros to 16) and its derivative.
__device__ __forceinline__ void basis16(float d, int K, float pi_over_rc, float pref, float* e, float* de,
                                        float& fc, float& dfc) {
    float s1, c1;
    sincospif(d * (pi_over_rc * 0.31830988618379067f), &s1, &c1);
    float inv_d = 1.0f / d;
    float sk = s1, skm1 = 0.f, ck = c1, ckm1 = 1.f;
#pragma unroll
    for (int k = 0; k < kKP; ++k) {
        bool on = k < K;
        e[k] = on ? pref * sk * inv_d : 0.f;
        if (de) de[k] = on ? pref * ((float)(k + 1) * pi_over_rc * ck - sk * inv_d) * inv_d : 0.f;
        float sn = 2.f * c1 * sk - skm1, cn = 2.f * c1 * ck - ckm1;
        skm1 = sk; sk = sn;
        ckm1 = ck; ck = cn;
    }
    fc = 0.5f * (c1 + 1.0f);
    dfc = -0.5f * pi_over_rc * s1;
}

// Stage a weight matrix as a K-major BF16 operand tile: B[n][k] = W[k][n]
// (transpose = true, W row-major [Kc][N]) or B[n][k] = W[n][k] (transpose =
// false, W row-major [N][Kc]); columns k >= Kreal are zero.
__device__ void stage_b(unsigned char* tile, const float* __restrict__ W, int N, int Kc, int Kreal, bool transpose) {
    for (int t = threadIdx.x; t < N * Kc; t += blockDim.x) {
        int n = t / Kc, k = t % Kc;
        float v = 0.f;
        if (k < Kreal) v = transpose ? __ldg(W + (size_t)k * N + n) : __ldg(W + (size_t)n * Kc + k);
        *reinterpret_cast<__nv_bfloat16*>(tile + tile_offset(n, k, Kc)) = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------------ per-atom tails (FP32)
template <int F>
__device__ __forceinline__ void stage_w_t(float* Ws, const float* __restrict__ Wg) {
    __syncthreads();
    for (int t = threadIdx.x; t < F * F; t += kT) Ws[(t / F) * (F + 1) + (t % F)] = __ldg(Wg + t);
    __syncthreads();
}

template <int F>
__device__ __forceinline__ float dot_t(const float* in_row, const float* Ws, int f, bool trans) {
    float acc = 0.f;
    if (trans) {
#pragma unroll 8
        for (int k = 0; k < F; ++k) acc += in_row[k] * Ws[f * (F + 1) + k];
    } else {
#pragma unroll 8
        for (int k = 0; k < F; ++k) acc += in_row[k] * Ws[k * (F + 1) + f];
    }
    return acc;
}

__device__ __forceinline__ float silu_acc(float a, float& sig) {
    sig = 1.0f / (1.0f + __expf(-a));
    return a * sig;
}

// Shared-memory layout (bytes) of the forward kernel.
template <int F>
struct FwdLayout {
    static constexpr int W1T = 0;                                 // [F][16] bf16
    static constexpr int W2T = W1T + F * kKP * 2;                 // [F][F] bf16
    static constexpr int B1 = W2T + F * F * 2;                    // [F] f32
    static constexpr int B2 = B1 + F * 4;                         // [F] f32
    static constexpr int A1 = B2 + F * 4;                         // [128][16] bf16
    static constexpr int A2 = A1 + kT * kKP * 2;                  // [128][F] bf16
    static constexpr int P = A2 + kT * F * 2;                     // [128][F+4] f32
    static constexpr int FC = P + kT * (F + 4) * 4;               // [128] f32
    static constexpr int J = FC + kT * 4;                         // [128] int
    static constexpr int ROW = J + kT * 4;                        // [128] int
    static constexpr int REP = ROW + kT * 4;                      // [128] f32
    static constexpr int MBAR = REP + kT * 4;                     // 8 B (+ taddr)
    static constexpr int ACC = MBAR + 16;                         // [A][F] f32
    static int bytes(int A) { return ACC + A * F * 4; }
};

template <int F>
__global__ void __launch_bounds__(kT) k_edge_fwd_bf16(PotArgs a, int K, int* status) {
    using L = FwdLayout<F>;
    extern __shared__ __align__(1024) unsigned char sm[];
    float* sb1 = reinterpret_cast<float*>(sm + L::B1);
    float* sb2 = reinterpret_cast<float*>(sm + L::B2);
    float* sP = reinterpret_cast<float*>(sm + L::P);
    float* sfc = reinterpret_cast<float*>(sm + L::FC);
    int* sj = reinterpret_cast<int*>(sm + L::J);
    int* srow = reinterpret_cast<int*>(sm + L::ROW);
    float* srep = reinterpret_cast<float*>(sm + L::REP);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L::MBAR);
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(sm + L::MBAR + 8);
    float* sAcc = reinterpret_cast<float*>(sm + L::ACC);
    constexpr int PS = F + 4;
    const int A = a.atoms_per_cta;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int l = a.layer;
    const int a0 = blockIdx.x * A;
    const int a1 = min(a.n_atoms, a0 + A);
    const int nA = a1 - a0;
    if (nA <= 0) return;

    stage_b(sm + L::W1T, a.P + a.off.W1[l], F, kKP, K, true);
    stage_b(sm + L::W2T, a.P + a.off.W2[l], F, F, F, true);
    for (int t = tid; t < F; t += kT) {
        sb1[t] = __ldg(a.P + a.off.b1[l] + t);
        sb2[t] = __ldg(a.P + a.off.b2[l] + t);
    }
    for (int t = tid; t < A * F; t += kT) sAcc[t] = 0.f;
    if (l == 0)
        for (int t = tid; t < nA; t += kT) a.erep[a0 + t] = 0.f;
    if (tid == 0) mbar_init(mbar, 1);
    if (warp == 0) tmem_alloc(taddr_s, 2 * F);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *taddr_s;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t idesc = idesc_bf16_f32(128, F);
    const uint32_t sA1 = smem_u32(sm + L::A1), sA2 = smem_u32(sm + L::A2);
    const uint32_t sW1T = smem_u32(sm + L::W1T), sW2T = smem_u32(sm + L::W2T);
    uint32_t phase = 0;
    bool ok = true;

    const long long e_beg = min((long long)a.row_ptr[a0], a.e_cap);
    const long long e_end = min((long long)a.row_ptr[a1], a.e_cap);
    int cur = -1;
    float run = 0.f;

    for (long long t0 = e_beg; t0 < e_end && ok; t0 += kT) {
        // ---- edge geometry and basis: one edge per thread
        {
            long long e = t0 + tid;
            float eb[kKP], fc = 0.f, dfc;
            if (e < e_end) {
                int j = a.col[e], i = a.recv[e];
                uint4 qi = a.q[i], qj = a.q[j];
                float3 r = edge_vec(qi, qj, a.frame[qi.w].qscale);
                float d = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
                basis16(d, K, a.pi_over_rc, a.bessel_pref, eb, nullptr, fc, dfc);
                sj[tid] = j;
                srow[tid] = i - a0;
                srep[tid] = l == 0 ? 0.5f * rep_phi(d, a.rep_a, a.rep_inv_rho, a.rep_rc, a.rep_pi_over_rc, nullptr) : 0.f;
            } else {
#pragma unroll
                for (int k = 0; k < kKP; ++k) eb[k] = 0.f;
                sj[tid] = a0;
                srow[tid] = -1;
                srep[tid] = 0.f;
            }
            sfc[tid] = fc;
            st_row8(sm + L::A1, tid, 0, kKP, eb);
            st_row8(sm + L::A1, tid, 8, kKP, eb + 8);
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            mma_bf16(tmem, make_desc(sA1, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
            mma_commit(mbar);
        }
        ok = mbar_wait(mbar, phase, kWaitIter);
        phase ^= 1;
        fence_after_sync();
        // ---- hidden = SiLU(D1 + b1) -> A2 (bf16)
#pragma unroll
        for (int c = 0; c < F; c += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float x = v[q] + sb1[c + q];
                v[q] = x * sigmoid_fast(x);
            }
            st_row8(sm + L::A2, tid, c, F, v);
            st_row8(sm + L::A2, tid, c + 8, F, v + 8);
        }
        fence_proxy_async();
        fence_before_sync();
        ok = __syncthreads_and(ok);
        fence_after_sync();
        if (tid == 0 && ok) {
#pragma unroll
            for (int kk = 0; kk < F / 16; ++kk)
                mma_bf16(tmem + F, make_desc(sA2 + kk * 256, 128, F * 16), make_desc(sW2T + kk * 256, 128, F * 16),
                         idesc, kk > 0);
            mma_commit(mbar);
        }
        ok = ok && mbar_wait(mbar, phase, kWaitIter);
        phase ^= 1;
        fence_after_sync();
        // ---- message w * u_j, w = fc (D2 + b2)
        {
            const float fc = sfc[tid];
            const float* uj = a.u + (size_t)sj[tid] * F;
#pragma unroll
            for (int c = 0; c < F; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + F + c, v);
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    float4 u4 = __ldg(reinterpret_cast<const float4*>(uj + c + q));
                    float4 m;
                    m.x = fc * (v[q] + sb2[c + q]) * u4.x;
                    m.y = fc * (v[q + 1] + sb2[c + q + 1]) * u4.y;
                    m.z = fc * (v[q + 2] + sb2[c + q + 2]) * u4.z;
                    m.w = fc * (v[q + 3] + sb2[c + q + 3]) * u4.w;
                    *reinterpret_cast<float4*>(sP + tid * PS + c + q) = m;
                }
            }
        }
        fence_before_sync();
        ok = __syncthreads_and(ok);
        // ---- row sums in edge order (thread F: pair repulsion energy)
        if (tid < F) {
            for (int e = 0; e < kT; ++e) {
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
            for (int e = 0; e < kT; ++e) {
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
        __syncthreads();   // the next tile rewrites srow, srep and sP
    }
    __syncthreads();
    if (tid < F && cur >= 0) sAcc[cur * F + tid] = run;
    if (tid == F && l == 0 && cur >= 0) a.erep[a0 + cur] = run;
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * F);
    if (!ok) {
        if (tid == 0) atomicOr(status, 1);
        return;
    }

    // ---------------- per-atom tail (FP32), scratch over A2 and P
    float* tX = reinterpret_cast<float*>(sm + L::A2);
    float* tY = tX + A * F;
    float* Ws = tY + A * F;
    const int f = tid % F, astep = kT / F;
    const bool last = (l == a.n_layers - 1);
    const float* P = a.P;
    for (int t = tid; t < nA * F; t += kT) tX[t] = sAcc[t];
    stage_w_t<F>(Ws, P + a.off.U1[l]);
    for (int r = tid / F; r < nA; r += astep) {
        float z = dot_t<F>(tX + r * F, Ws, f, false) + __ldg(P + a.off.c1[l] + f);
        a.z[(size_t)(a0 + r) * F + f] = z;
        float sg;
        tY[r * F + f] = silu_acc(z, sg);
    }
    stage_w_t<F>(Ws, P + a.off.U2[l]);
    for (int r = tid / F; r < nA; r += astep) {
        size_t o = (size_t)(a0 + r) * F + f;
        float hn = a.h[o] + dot_t<F>(tY + r * F, Ws, f, false) + __ldg(P + a.off.c2[l] + f);
        a.h[o] = hn;
        tX[r * F + f] = hn;
    }
    if (!last) {
        stage_w_t<F>(Ws, P + a.off.W_in[l + 1]);
        for (int r = tid / F; r < nA; r += astep)
            a.u_next[(size_t)(a0 + r) * F + f] = dot_t<F>(tX + r * F, Ws, f, false);
        return;
    }
    stage_w_t<F>(Ws, P + a.off.R1);
    for (int r = tid / F; r < nA; r += astep) {
        float qv = dot_t<F>(tX + r * F, Ws, f, false) + __ldg(P + a.off.d1 + f);
        float sg;
        float s = silu_acc(qv, sg);
        float r2 = __ldg(P + a.off.R2 + f);
        tY[r * F + f] = sg * (1.f + qv * (1.f - sg)) * r2;
        sAcc[r * F + f] = s * r2;
    }
    __syncthreads();
    for (int r = tid; r < nA; r += kT) {
        double e = 0.0;
        for (int k = 0; k < F; ++k) e += (double)sAcc[r * F + k];
        int i = a0 + r;
        e += (double)__ldg(P + a.off.d2) + (double)__ldg(P + a.off.e0 + a.species[i]);
        e += (double)a.erep[i];
        a.Ei[i] = e;
    }
    for (int r = tid / F; r < nA; r += astep) {
        float g = dot_t<F>(tY + r * F, Ws, f, true);
        a.gh[(size_t)(a0 + r) * F + f] = g;
        tX[r * F + f] = g;
    }
    stage_w_t<F>(Ws, P + a.off.U2[l]);
    for (int r = tid / F; r < nA; r += astep) {
        float gy = dot_t<F>(tX + r * F, Ws, f, true);
        float z = a.z[(size_t)(a0 + r) * F + f];
        float sg;
        (void)silu_acc(z, sg);
        tY[r * F + f] = gy * sg * (1.f + z * (1.f - sg));
    }
    stage_w_t<F>(Ws, P + a.off.U1[l]);
    for (int r = tid / F; r < nA; r += astep)
        a.mbar_out[(size_t)(a0 + r) * F + f] = dot_t<F>(tY + r * F, Ws, f, true);
}

// ------------------------------------------------------------ backward
template <int F>
struct BwdLayout {
    static constexpr int W1T = 0;                                 // [F][16] bf16, B[n][k] = W1[k][n]
    static constexpr int W2T = W1T + F * kKP * 2;                 // [F][F] bf16, B[n][k] = W2[k][n]
    static constexpr int W2N = W2T + F * F * 2;                   // [F][F] bf16, B[n][k] = W2[n][k]
    static constexpr int B1 = W2N + F * F * 2;                    // [F] f32
    static constexpr int B2 = B1 + F * 4;                         // [F] f32
    static constexpr int A1 = B2 + F * 4;                         // [128][16] bf16 basis
    static constexpr int A4 = A1 + kT * kKP * 2;                  // [128][16] bf16 basis derivative
    static constexpr int A2 = A4 + kT * kKP * 2;                  // [128][F] bf16: SiLU hidden, then g
    static constexpr int P = A2 + kT * F * 2;                     // [128][F+4] f32 ubar messages
    static constexpr int J = P + kT * (F + 4) * 4;                // [128] int
    static constexpr int ROW = J + kT * 4;                        // [128] int
    static constexpr int SLOT = ROW + kT * 4;                     // [4][32][12] f32 warp partials
    static constexpr int NSLOT = SLOT + 4 * 32 * 12 * 4;          // [4] int
    static constexpr int MBAR = NSLOT + 16;                       // mbar + taddr
    static constexpr int ACC = MBAR + 16;                         // [A][F] ubar
    static int bytes(int A) { return ACC + A * F * 4 + A * 4 * 4 + A * 8 * 4; }
};

template <int F>
__global__ void __launch_bounds__(kT) k_edge_bwd_bf16(PotArgs a, int K, int* status) {
    using L = BwdLayout<F>;
    extern __shared__ __align__(1024) unsigned char sm[];
    float* sb1 = reinterpret_cast<float*>(sm + L::B1);
    float* sb2 = reinterpret_cast<float*>(sm + L::B2);
    float* sP = reinterpret_cast<float*>(sm + L::P);
    int* sj = reinterpret_cast<int*>(sm + L::J);
    int* srow = reinterpret_cast<int*>(sm + L::ROW);
    float* slot = reinterpret_cast<float*>(sm + L::SLOT);
    int* nslot = reinterpret_cast<int*>(sm + L::NSLOT);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L::MBAR);
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(sm + L::MBAR + 8);
    const int A = a.atoms_per_cta;
    float* sAcc = reinterpret_cast<float*>(sm + L::ACC);
    float* sF = sAcc + A * F;      // [A][4]
    float* sV = sF + A * 4;        // [A][8]
    constexpr int PS = F + 4;
    constexpr int TCOLS = 4 * F;   // D1 | D4 | D2 | D3
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int l = a.layer;
    const int a0 = blockIdx.x * A;
    const int a1 = min(a.n_atoms, a0 + A);
    const int nA = a1 - a0;
    if (nA <= 0) return;
    const bool need_ubar = (l > 0);

    stage_b(sm + L::W1T, a.P + a.off.W1[l], F, kKP, K, true);
    stage_b(sm + L::W2T, a.P + a.off.W2[l], F, F, F, true);
    stage_b(sm + L::W2N, a.P + a.off.W2[l], F, F, F, false);
    for (int t = tid; t < F; t += kT) {
        sb1[t] = __ldg(a.P + a.off.b1[l] + t);
        sb2[t] = __ldg(a.P + a.off.b2[l] + t);
    }
    for (int t = tid; t < A * F; t += kT) sAcc[t] = 0.f;
    for (int t = tid; t < A * 12; t += kT) sF[t] = 0.f;
    if (tid == 0) mbar_init(mbar, 1);
    if (warp == 0) tmem_alloc(taddr_s, TCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *taddr_s;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t tD1 = tmem, tD4 = tmem + F, tD2 = tmem + 2 * F, tD3 = tmem + 3 * F;
    const uint32_t idesc = idesc_bf16_f32(128, F);
    const uint32_t sA1 = smem_u32(sm + L::A1), sA4 = smem_u32(sm + L::A4), sA2 = smem_u32(sm + L::A2);
    const uint32_t sW1T = smem_u32(sm + L::W1T), sW2T = smem_u32(sm + L::W2T), sW2N = smem_u32(sm + L::W2N);
    uint32_t phase = 0;
    bool ok = true;

    const long long e_beg = min((long long)a.row_ptr[a0], a.e_cap);
    const long long e_end = min((long long)a.row_ptr[a1], a.e_cap);
    int cur = -1;          // running row of the ubar sums (threads < F) and force sums (threads F..F+8)
    float run = 0.f;

    for (long long t0 = e_beg; t0 < e_end && ok; t0 += kT) {
        long long e = t0 + tid;
        const bool valid = e < e_end;
        int j = a0, row = -1;
        float fc = 0.f, dfc = 0.f, d = 1.f, rx = 0.f, ry = 0.f, rz = 0.f;
        {
            float eb[kKP], db[kKP];
            if (valid) {
                j = a.col[e];
                int i = a.recv[e];
                row = i - a0;
                uint4 qi = a.q[i], qj = a.q[j];
                float3 r = edge_vec(qi, qj, a.frame[qi.w].qscale);
                d = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
                float inv = 1.0f / d;
                rx = r.x * inv; ry = r.y * inv; rz = r.z * inv;
                basis16(d, K, a.pi_over_rc, a.bessel_pref, eb, db, fc, dfc);
            } else {
#pragma unroll
                for (int k = 0; k < kKP; ++k) { eb[k] = 0.f; db[k] = 0.f; }
            }
            sj[tid] = j;
            srow[tid] = row;
            st_row8(sm + L::A1, tid, 0, kKP, eb);
            st_row8(sm + L::A1, tid, 8, kKP, eb + 8);
            st_row8(sm + L::A4, tid, 0, kKP, db);
            st_row8(sm + L::A4, tid, 8, kKP, db + 8);
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            mma_bf16(tD1, make_desc(sA1, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
            mma_bf16(tD4, make_desc(sA4, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
            mma_commit(mbar);
        }
        ok = mbar_wait(mbar, phase, kWaitIter);
        phase ^= 1;
        fence_after_sync();
        // ---- A2 = SiLU(D1 + b1)
#pragma unroll
        for (int c = 0; c < F; c += 16) {
            float v[16];
            tmem_ld16(tD1 + lane_base + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float x = v[q] + sb1[c + q];
                v[q] = x * sigmoid_fast(x);
            }
            st_row8(sm + L::A2, tid, c, F, v);
            st_row8(sm + L::A2, tid, c + 8, F, v + 8);
        }
        fence_proxy_async();
        fence_before_sync();
        ok = __syncthreads_and(ok);
        fence_after_sync();
        if (tid == 0 && ok) {
#pragma unroll
            for (int kk = 0; kk < F / 16; ++kk)
                mma_bf16(tD2, make_desc(sA2 + kk * 256, 128, F * 16), make_desc(sW2T + kk * 256, 128, F * 16),
                         idesc, kk > 0);
            mma_commit(mbar);
        }
        ok = ok && mbar_wait(mbar, phase, kWaitIter);
        phase ^= 1;
        fence_after_sync();
        // ---- phi = D2 + b2; g = mbar_i u_j + mbar_j u_i -> A2 (bf16); g . phi; ubar message
        float gphi = 0.f;
        {
            const int i = row < 0 ? a0 : a0 + row;
            const float* uj = a.u + (size_t)j * F;
            const float* mj = a.mbar + (size_t)j * F;
            const float* ui = a.u + (size_t)i * F;
            const float* mi = a.mbar + (size_t)i * F;
#pragma unroll
            for (int c = 0; c < F; c += 16) {
                float v[16], g[16];
                tmem_ld16(tD2 + lane_base + c, v);
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    float4 u4 = __ldg(reinterpret_cast<const float4*>(uj + c + q));
                    float4 m4 = __ldg(reinterpret_cast<const float4*>(mj + c + q));
                    float4 ui4 = __ldg(reinterpret_cast<const float4*>(ui + c + q));
                    float4 mi4 = __ldg(reinterpret_cast<const float4*>(mi + c + q));
                    float ph0 = v[q] + sb2[c + q], ph1 = v[q + 1] + sb2[c + q + 1];
                    float ph2 = v[q + 2] + sb2[c + q + 2], ph3 = v[q + 3] + sb2[c + q + 3];
                    g[q] = mi4.x * u4.x + m4.x * ui4.x;
                    g[q + 1] = mi4.y * u4.y + m4.y * ui4.y;
                    g[q + 2] = mi4.z * u4.z + m4.z * ui4.z;
                    g[q + 3] = mi4.w * u4.w + m4.w * ui4.w;
                    gphi += g[q] * ph0 + g[q + 1] * ph1 + g[q + 2] * ph2 + g[q + 3] * ph3;
                    if (need_ubar)
                        *reinterpret_cast<float4*>(sP + tid * PS + c + q) =
                            make_float4(fc * ph0 * m4.x, fc * ph1 * m4.y, fc * ph2 * m4.z, fc * ph3 * m4.w);
                }
                st_row8(sm + L::A2, tid, c, F, g);
                st_row8(sm + L::A2, tid, c + 8, F, g + 8);
            }
        }
        fence_proxy_async();
        fence_before_sync();
        ok = __syncthreads_and(ok);
        fence_after_sync();
        if (tid == 0 && ok) {
#pragma unroll
            for (int kk = 0; kk < F / 16; ++kk)
                mma_bf16(tD3, make_desc(sA2 + kk * 256, 128, F * 16), make_desc(sW2N + kk * 256, 128, F * 16),
                         idesc, kk > 0);
            mma_commit(mbar);
        }
        ok = ok && mbar_wait(mbar, phase, kWaitIter);
        phase ^= 1;
        fence_after_sync();
        // ---- dE/dd = fc' (g . phi) + fc sum_k D3_k SiLU'(a_k) D4_k (+ repulsion on layer 0)
        float s2 = 0.f;
#pragma unroll
        for (int c = 0; c < F; c += 16) {
            float ab[16], av[16], tv[16];
            tmem_ld16(tD3 + lane_base + c, ab);
            tmem_ld16(tD1 + lane_base + c, av);
            tmem_ld16(tD4 + lane_base + c, tv);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float x = av[q] + sb1[c + q];
                float sg = sigmoid_fast(x);
                s2 += ab[q] * (sg * (1.f + x * (1.f - sg))) * tv[q];
            }
        }
        float se = dfc * gphi + fc * s2;
        if (l == 0 && valid) {
            float dphi;
            (void)rep_phi(d, a.rep_a, a.rep_inv_rho, a.rep_rc, a.rep_pi_over_rc, &dphi);
            se += dphi;
        }
        // ---- force (3) and virial (6) per edge: warp segmented scan, then per-row partials
        {
            float val[9];
            val[0] = se * rx; val[1] = se * ry; val[2] = se * rz;
            float hv = -0.5f * se * d;
            val[3] = hv * rx * rx; val[4] = hv * ry * ry; val[5] = hv * rz * rz;
            val[6] = hv * rx * ry; val[7] = hv * rx * rz; val[8] = hv * ry * rz;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int ro = __shfl_up_sync(0xffffffffu, row, off);
                bool same = lane >= off && ro == row;
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    float y = __shfl_up_sync(0xffffffffu, val[c], off);
                    if (same) val[c] += y;
                }
            }
            int rn = __shfl_down_sync(0xffffffffu, row, 1);
            bool seg_end = row >= 0 && (lane == 31 || rn != row);
            unsigned int ends = __ballot_sync(0xffffffffu, seg_end);
            if (seg_end) {
                int k = __popc(ends & ((1u << lane) - 1u));
                float* o = slot + (warp * 32 + k) * 12;
                o[0] = __int_as_float(row);
#pragma unroll
                for (int c = 0; c < 9; ++c) o[1 + c] = val[c];
            }
            if (lane == 0) nslot[warp] = __popc(ends);
        }
        fence_before_sync();
        ok = __syncthreads_and(ok);
        // ---- combine in edge order: ubar row sums (threads < F), force/virial (threads F..F+8)
        if (need_ubar && tid < F) {
            for (int ee = 0; ee < kT; ++ee) {
                int r = srow[ee];
                if (r < 0) break;
                if (r != cur) {
                    if (cur >= 0) sAcc[cur * F + tid] = run;
                    cur = r;
                    run = 0.f;
                }
                run += sP[ee * PS + tid];
            }
        } else if (tid >= F && tid < F + 9) {
            const int c = tid - F;
            for (int w = 0; w < 4; ++w) {
                const int ns = nslot[w];
                for (int k = 0; k < ns; ++k) {
                    const float* o = slot + (w * 32 + k) * 12;
                    int r = __float_as_int(o[0]);
                    if (r != cur) {
                        if (cur >= 0) {
                            if (c < 3) sF[cur * 4 + c] = run;
                            else sV[cur * 8 + c - 3] = run;
                        }
                        cur = r;
                        run = 0.f;
                    }
                    run += o[1 + c];
                }
            }
        }
        __syncthreads();   // the next tile rewrites srow, sP and the slots
    }
    __syncthreads();
    if (cur >= 0) {
        if (need_ubar && tid < F) sAcc[cur * F + tid] = run;
        else if (tid >= F && tid < F + 9) {
            const int c = tid - F;
            if (c < 3) sF[cur * 4 + c] = run;
            else sV[cur * 8 + c - 3] = run;
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
    if (!ok) {
        if (tid == 0) atomicOr(status, 1);
        return;
    }
    for (int t = tid; t < nA * 3; t += kT) {
        int r = t / 3, c = t % 3;
        size_t o = (size_t)c * a.n_atoms + a0 + r;
        a.force[o] = a.accumulate ? a.force[o] + sF[r * 4 + c] : sF[r * 4 + c];
    }
    for (int t = tid; t < nA * 6; t += kT) {
        int r = t / 6, c = t % 6;
        size_t o = (size_t)(a0 + r) * 6 + c;
        a.vir6[o] = a.accumulate ? a.vir6[o] + sV[r * 8 + c] : sV[r * 8 + c];
    }
    if (!need_ubar) return;
    float* tX = reinterpret_cast<float*>(sm + L::A2);
    float* tY = tX + A * F;
    float* Ws = tY + A * F;
    const int f = tid % F, astep = kT / F;
    const float* P = a.P;
    for (int t = tid; t < nA * F; t += kT) tX[t] = sAcc[t];
    stage_w_t<F>(Ws, P + a.off.W_in[l]);
    for (int r = tid / F; r < nA; r += astep) {
        size_t o = (size_t)(a0 + r) * F + f;
        float g = a.gh[o] + dot_t<F>(tX + r * F, Ws, f, true);
        a.gh[o] = g;
        tY[r * F + f] = g;
    }
    stage_w_t<F>(Ws, P + a.off.U2[l - 1]);
    for (int r = tid / F; r < nA; r += astep) {
        float gy = dot_t<F>(tY + r * F, Ws, f, true);
        float z = a.z_prev[(size_t)(a0 + r) * F + f];
        float sg;
        (void)silu_acc(z, sg);
        tX[r * F + f] = gy * sg * (1.f + z * (1.f - sg));
    }
    stage_w_t<F>(Ws, P + a.off.U1[l - 1]);
    for (int r = tid / F; r < nA; r += astep)
        a.mbar_out[(size_t)(a0 + r) * F + f] = dot_t<F>(tX + r * F, Ws, f, true);
}

template <int F>
int fwd_max_atoms() {
    // tail scratch 2 A F + F (F + 1) floats must fit in the A2 + P region
    const int region = (FwdLayout<F>::FC - FwdLayout<F>::A2) / 4;
    int best = 0;
    for (int A = 8; A <= 256; A += 8)
        if (2 * A * F + F * (F + 1) <= region && FwdLayout<F>::bytes(A) <= 227 * 1024) best = A;
    return best;
}

template <int F>
int bwd_max_atoms() {
    const int region = (BwdLayout<F>::J - BwdLayout<F>::A2) / 4;
    int best = 0;
    for (int A = 8; A <= 256; A += 8)
        if (2 * A * F + F * (F + 1) <= region && BwdLayout<F>::bytes(A) <= 227 * 1024) best = A;
    return best;
}

template <int F>
void fwd_go(const PotArgs& a, int K, int* status, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_edge_fwd_bf16<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    k_edge_fwd_bf16<F><<<grid, kT, FwdLayout<F>::bytes(a.atoms_per_cta), s>>>(a, K, status);
}

template <int F>
void bwd_go(const PotArgs& a, int K, int* status, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_edge_bwd_bf16<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    k_edge_bwd_bf16<F><<<grid, kT, BwdLayout<F>::bytes(a.atoms_per_cta), s>>>(a, K, status);
}

}  // namespace

void launch_edge_fwd_bf16(const PotArgs& a, int F, int K, int* status, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    if (F == 64) fwd_go<64>(a, K, status, s);
    else fwd_go<32>(a, K, status, s);
    count_launch();
}

void launch_edge_bwd_bf16(const PotArgs& a, int F, int K, int* status, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    if (F == 64) bwd_go<64>(a, K, status, s);
    else bwd_go<32>(a, K, status, s);
    count_launch();
}

int max_atoms_per_cta_bf16(int F, bool bwd) {
    if (F == 64) return bwd ? bwd_max_atoms<64>() : fwd_max_atoms<64>();
    if (F == 32) return bwd ? bwd_max_atoms<32>() : fwd_max_atoms<32>();
    return 0;
}

}  // namespace dmts
