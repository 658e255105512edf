// Distillation gradient of a single-layer model (hand-written adjoints): the
// parameter gradient of the energy and force loss
//   L(theta) = 1/M sum_frames [ lambda_E ((E(theta) - E_ref) / N)^2
//                               + 1/(3 N) sum_i |F_i(theta) - F_ref,i|^2 ]
// (lambda_E = 0: force matching), the forces F = -dE/dx making it a second
// derivative of the energy.
//
// With g = dL/dF = 2 (F - F_ref) / (3 N M) per frame and
//   Psi(theta) = sum_i g_i . dE/dx_i = d/d eps E(x + eps g) |_{eps=0},
// dL/dtheta = -dPsi/dtheta. Psi is the directional derivative of the energy
// along x' = g, so it is the energy's forward pass carried with tangents:
// only the pair distances move, d' = delta_ij = rhat_ij . (g_j - g_i), hence
//   w'_ij = delta_ij dw/dd = delta (fc' phi + fc (SiLU'(a) * (e' W1)) W2),
//   m'_i = sum_j w'_ij * u_j,  z' = m' U1,  h1' = (SiLU'(z) * z') U2,
//   q' = h1' R1,  Psi = sum_i (SiLU'(q_i) * q'_i) . R2.
// The kernels below take the reverse of this tangent graph with respect to
// theta: a tangent edge pass (m'), a per-atom adjoint pass (dPsi/dm,
// dPsi/dm' and the per-atom weight gradients), and an edge pass for the
// filter-weight gradients and dPsi/du. Every gradient is summed per CTA and
// the CTA partials are added in a fixed order (deterministic). The FP32 mode
// runs every step in FP32 on the SIMT pipes; in the BF16 mode the two edge
// passes run their per-pair MLP products and their weight-gradient sums over
// pairs on the tensor cores (BF16 operands, FP32 accumulation in tensor
// memory), the per-atom pass stays FP32.
//
// The energy term adds c_E dE/dtheta per frame, c_E = dL/dE = 2 lambda_E
// (E - E_ref) / (M N^2): the same reverse pass seeded at the readout with
// -c_E besides the tangent's seed (the passes accumulate -d(.)/dtheta), so
// dPsi/dq gains -c_E SiLU'(q) R2, dPsi/dR2 gains -c_E SiLU(q), and d2 and
// e0[Z_i] gain -c_E per atom.
#include <algorithm>
#include <initializer_list>
#include <utility>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "umma.cuh"

namespace dmts {

namespace {

using namespace umma;

constexpr int kT = 256;
constexpr int kFmAtomsMax = 96;              // atoms per CTA of the edge passes, at most
constexpr uint32_t kFmWait = 1u << 22;       // bounded mbarrier polls (tensor-core weight gradients)

__device__ __forceinline__ float sgm(float x) { return 1.0f / (1.0f + expf(-x)); }
// SiLU, its first and second derivatives at a
__device__ __forceinline__ void silu3(float a, float& s, float& d1, float& d2) {
    float g = sgm(a);
    s = a * g;
    d1 = g * (1.f + a * (1.f - g));
    d2 = g * (1.f - g) * (2.f + a * (1.f - 2.f * g));
}

template <int K>
__device__ __forceinline__ void basis_pair(float d, float pi_over_rc, float pref, float* e, float* de, float& fc,
                                           float& dfc) {
    float s1, c1;
    sincospif(d * (pi_over_rc * 0.31830988618379067f), &s1, &c1);
    float inv_d = 1.0f / d;
    float sk = s1, skm1 = 0.f, ck = c1, ckm1 = 1.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float kw = (float)(k + 1) * pi_over_rc;
        e[k] = pref * sk * inv_d;
        de[k] = pref * (kw * ck - sk * inv_d) * inv_d;
        float sn = 2.f * c1 * sk - skm1, cn = 2.f * c1 * ck - ckm1;
        skm1 = sk; sk = sn;
        ckm1 = ck; ck = cn;
    }
    fc = 0.5f * (c1 + 1.0f);
    dfc = -0.5f * pi_over_rc * s1;
}

// ------------------------------------------------------------ residual g
// g_i = c (F_i - F_ref,i) (SoA), c = 2 / (3 N M); per-atom squared residual
// (FP64) for the loss.
__global__ void k_fm_residual(int n, const float* __restrict__ f, const double* __restrict__ f_ref_aos, double c,
                              float* __restrict__ g, double* __restrict__ sq) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double r = (double)f[(size_t)k * n + i] - f_ref_aos[3 * (size_t)i + k];
        g[(size_t)k * n + i] = (float)(c * r);
        s += r * r;
    }
    sq[i] = s;
}

// ------------------------------------------------------------ edge tile (shared by both edge passes)
// One CTA owns atoms [a0, a0 + A) and walks their CSR edges in tiles of TE
// edges; thread (eg, fg) owns edges 4eg..4eg+3 and features 4fg..4fg+3 of
// every [TE x F] tile.
template <int F, int K>
struct Geo {
    static constexpr int TE = 4096 / F;
    static constexpr int FG = F / 4;
};

// acc[r][c] = sum_k AT[k][e0 + r] W[k][f0 + c]
template <int KIN, int TE, int F>
__device__ __forceinline__ void tgemm(const float* AT, const float* W, int e0, int f0, float acc[4][4]) {
#pragma unroll 8
    for (int k = 0; k < KIN; ++k) {
        float4 x = *reinterpret_cast<const float4*>(AT + k * TE + e0);
        float4 w = *reinterpret_cast<const float4*>(W + k * F + f0);
        float xa[4] = {x.x, x.y, x.z, x.w}, wf[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] += xa[r] * wf[c];
    }
}

template <int TE>
__device__ __forceinline__ void store_tT(float* T, int f0, int e0, const float v[4][4]) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(T + (f0 + c) * TE + e0) = make_float4(v[0][c], v[1][c], v[2][c], v[3][c]);
}

// Shared-memory carve of both edge passes (floats).
template <int F, int K>
struct EdgeSmem {
    static constexpr int TE = Geo<F, K>::TE;
    float W1[K * F], b1[F], W2[F * F], W2T[F * F], b2[F];
    float BT[K * TE], DT[K * TE];        // basis, derivative, transposed
    float ST[F * TE], PT[F * TE];        // SiLU(a), SiLU'(a) * T  (transposed)
    float X[TE * (F + 4)], Y[TE * (F + 4)];   // per-edge rows (msg, phibar, gbar, abar, tbar)
    float fc[TE], dfc[TE], delta[TE];
    int j[TE], row[TE];
    float acc[kFmAtomsMax * F];          // per-atom row sums of the CTA
    float slot[kT / 32][2][F];           // per-warp open row segments of a tile (row_sums)
    int slot_row[kT / 32][2];
};

// ---------------------------------------------------------------- tensor-core operands (BF16 mode)
// In the BF16 mode the per-pair MLP products of both edge passes and the
// filter-weight gradient sums over pairs run on tcgen05: BF16 operands
// (K-major, no swizzle, umma.cuh), FP32 accumulators in tensor memory, the
// rest FP32 as in the passes above. A tile's TE = 128 pairs are the 128
// lanes of tensor memory (pair e in lane e). Per tile:
//   MMA1  [a - b1 | T]   = [e | e'] W1                    (N = F each, K = 16: e padded)
//   MMA2  [phi - b2 | q] = [SiLU(a) | SiLU'(a) T] W2      (K = F)
//   MMA3  [sb | pb]      = [phibar | gbar] W2^T            (gradient pass)
// and the weight gradients, summed over the CTA's tiles: an A operand of 128
// rows by the tile's pairs (the ST and PT region, 32 KB) holds SiLU(a)^T
// (rows 0-31), (SiLU'(a) T)^T (32-63), e^T and e'^T (K rows each), zero
// rows and a row of ones (127); B holds [phibar | gbar], later
// [abar | tbar], as 64 rows by the pairs; D1 += A B1^T, D2 += A B2^T (64
// FP32 columns each), and
//   dW2[k][f] = D1[k][f] + D1[32 + k][32 + f],   db2[f] = D1[127][f],
//   dW1[k][f] = D2[64 + k][f] + D2[64 + K + k][32 + f],   db1[f] = D2[127][f]
// (the other blocks of D1 and D2 are products nobody reads). Accumulator
// pairs are read back by all eight warps into FP32 rows [TE][F + 4], which
// the 4 x 4 thread blocks of the passes read as before.
constexpr int kKb = 16;                      // basis columns of the MMA1 operands (one K step)
constexpr uint32_t kBf16Ones = 0x3F803F80u;  // two BF16 ones

template <int F>
struct TcWeights {
    unsigned char w1t[F * kKb * 2];          // B[n][k] = W1[k][n] (zero for k >= K)
    unsigned char w2t[F * F * 2];            // B[n][k] = W2[k][n]
    unsigned char w2n[F * F * 2];            // B[n][k] = W2[n][k]
};

// Tangent pass: the MMA1 and MMA2 operands sit in the ST and PT region,
// which this pass does not otherwise use.
template <int F, int K>
struct TangTc {
    EdgeSmem<F, K> e;
    TcWeights<F> w;
    uint64_t mbar;
    uint32_t taddr;
};

template <int F, int K>
struct GradTc {
    static constexpr int TE = Geo<F, K>::TE;
    EdgeSmem<F, K> e;                        // ST and PT: the weight-gradient A operand
    TcWeights<F> w;
    unsigned char a1[2][TE * kKb * 2];       // e | e' (pair rows)
    unsigned char a2[2][TE * F * 2];         // SiLU(a) | SiLU'(a) T
    unsigned char a3[2][TE * F * 2];         // phibar | gbar
    unsigned char b[64 * TE * 2];            // weight-gradient B operand
    float Z[2][TE * (F + 4)];                // MMA2 and MMA3 results as FP32 rows
    uint64_t mbar;
    uint32_t taddr;
};

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Four consecutive pairs (k = e0 .. e0 + 3, e0 a multiple of 4) of operand
// row r as BF16 (one 8-byte store).
__device__ __forceinline__ void st_k4(unsigned char* tile, int r, int e0, int Kc, float v0, float v1, float v2,
                                      float v3) {
    *reinterpret_cast<uint2*>(tile + tile_offset(r, e0, Kc)) = make_uint2(bf16x2(v0, v1), bf16x2(v2, v3));
}

template <int F, int K>
__device__ __forceinline__ void load_weights(EdgeSmem<F, K>& S, const PotArgs& a) {
    for (int t = threadIdx.x; t < K * F; t += kT) S.W1[t] = __ldg(a.P + a.off.W1[0] + t);
    for (int t = threadIdx.x; t < F * F; t += kT) {
        float w = __ldg(a.P + a.off.W2[0] + t);
        S.W2[t] = w;
        S.W2T[(t % F) * F + t / F] = w;
    }
    for (int t = threadIdx.x; t < F; t += kT) {
        S.b1[t] = __ldg(a.P + a.off.b1[0] + t);
        S.b2[t] = __ldg(a.P + a.off.b2[0] + t);
    }
}

// One pair's inputs: its atoms, their fixed-point positions and residual
// rows g (threads < TE; loaded a tile ahead by the tensor-core passes).
struct PairIn {
    int j = 0, i = 0;
    bool valid = false;
    uint4 qi, qj;
    float gi[3], gj[3];
};

__device__ __forceinline__ void pair_idx(const PotArgs& a, long long e, long long e_end, PairIn& p) {
    p.valid = e < e_end;
    if (p.valid) {
        p.j = DMTS_IDX(a.col[e], a.n_atoms, a.check);
        p.i = DMTS_IDX(a.recv[e], a.n_atoms, a.check);
    }
}

__device__ __forceinline__ void pair_pos(const PotArgs& a, const float* __restrict__ g, PairIn& p) {
    if (p.valid) {
        const int n = a.n_atoms;
        p.qi = a.q[p.i];
        p.qj = a.q[p.j];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p.gi[c] = g[c * n + p.i];
            p.gj[c] = g[c * n + p.j];
        }
    }
}

// Per-edge setup of pair tid (threads < TE) from its inputs: geometry, basis,
// delta = rhat . (g_j - g_i); a1 (tensor-core passes, else null): e and e'
// also as the BF16 pair rows of the MMA1 operands (16 columns, zero past K).
template <int F, int K>
__device__ __forceinline__ void edge_setup_in(EdgeSmem<F, K>& S, const PotArgs& a, const PairIn& p, int a0,
                                              unsigned char* a1) {
    constexpr int TE = Geo<F, K>::TE;
    const int tid = threadIdx.x;
    float eb[K], db[K];
    if (p.valid) {
        float3 r = edge_vec(p.qi, p.qj, a.frame[p.qi.w].qscale);
        float d = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
        float inv = 1.0f / d;
        float fc, dfc;
        basis_pair<K>(d, a.pi_over_rc, a.bessel_pref, eb, db, fc, dfc);
        float dl = (r.x * (p.gj[0] - p.gi[0]) + r.y * (p.gj[1] - p.gi[1]) + r.z * (p.gj[2] - p.gi[2])) * inv;
        S.fc[tid] = fc;
        S.dfc[tid] = dfc;
        S.delta[tid] = dl;
        S.j[tid] = p.j;
        S.row[tid] = p.i - a0;
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) { eb[k] = 0.f; db[k] = 0.f; }
        S.fc[tid] = 0.f;
        S.dfc[tid] = 0.f;
        S.delta[tid] = 0.f;
        S.j[tid] = a0;
        S.row[tid] = -1;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        S.BT[k * TE + tid] = eb[k];
        S.DT[k * TE + tid] = db[k];
    }
    if (a1) {
        static_assert(K <= kKb && K % 8 == 0, "whole 8-column chunks of the basis");
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += 8) {
            *reinterpret_cast<uint4*>(a1 + tile_offset(tid, k0, kKb)) =
                make_uint4(bf16x2(eb[k0], eb[k0 + 1]), bf16x2(eb[k0 + 2], eb[k0 + 3]),
                           bf16x2(eb[k0 + 4], eb[k0 + 5]), bf16x2(eb[k0 + 6], eb[k0 + 7]));
            *reinterpret_cast<uint4*>(a1 + TE * kKb * 2 + tile_offset(tid, k0, kKb)) =
                make_uint4(bf16x2(db[k0], db[k0 + 1]), bf16x2(db[k0 + 2], db[k0 + 3]),
                           bf16x2(db[k0 + 4], db[k0 + 5]), bf16x2(db[k0 + 6], db[k0 + 7]));
        }
#pragma unroll
        for (int k0 = K; k0 < kKb; k0 += 8) {
            *reinterpret_cast<uint4*>(a1 + tile_offset(tid, k0, kKb)) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(a1 + TE * kKb * 2 + tile_offset(tid, k0, kKb)) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// The same with the pair's inputs loaded here (the FP32 passes; written out
// so that their register allocation stays that of a single load-and-compute).
template <int F, int K>
__device__ __forceinline__ void edge_setup(EdgeSmem<F, K>& S, const PotArgs& a, const float* __restrict__ g,
                                           long long t0, long long e_end, int a0) {
    constexpr int TE = Geo<F, K>::TE;
    const int tid = threadIdx.x;
    if (tid >= TE) return;
    long long e = t0 + tid;
    float eb[K], db[K];
    if (e < e_end) {
        int j = DMTS_IDX(a.col[e], a.n_atoms, a.check), i = DMTS_IDX(a.recv[e], a.n_atoms, a.check);
        uint4 qi = a.q[i], qj = a.q[j];
        float3 r = edge_vec(qi, qj, a.frame[qi.w].qscale);
        float d = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
        float inv = 1.0f / d;
        float fc, dfc;
        basis_pair<K>(d, a.pi_over_rc, a.bessel_pref, eb, db, fc, dfc);
        const int n = a.n_atoms;
        float dl = (r.x * (g[j] - g[i]) + r.y * (g[n + j] - g[n + i]) + r.z * (g[2 * n + j] - g[2 * n + i])) * inv;
        S.fc[tid] = fc;
        S.dfc[tid] = dfc;
        S.delta[tid] = dl;
        S.j[tid] = j;
        S.row[tid] = i - a0;
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) { eb[k] = 0.f; db[k] = 0.f; }
        S.fc[tid] = 0.f;
        S.dfc[tid] = 0.f;
        S.delta[tid] = 0.f;
        S.j[tid] = a0;
        S.row[tid] = -1;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        S.BT[k * TE + tid] = eb[k];
        S.DT[k * TE + tid] = db[k];
    }
}

// a = e W1 + b1, T = e' W1: writes SiLU(a) to ST and SiLU'(a) T to PT; keeps
// SiLU'(a), SiLU''(a) and T of the thread's [4 x 4] block.
template <int F, int K>
__device__ __forceinline__ void filter_hidden(EdgeSmem<F, K>& S, int e0, int f0, float sp[4][4], float spp[4][4],
                                              float tt[4][4]) {
    constexpr int TE = Geo<F, K>::TE;
    float av[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) { av[r][c] = S.b1[f0 + c]; tt[r][c] = 0.f; }
    tgemm<K, TE, F>(S.BT, S.W1, e0, f0, av);
    tgemm<K, TE, F>(S.DT, S.W1, e0, f0, tt);
    float s[4][4], p[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            silu3(av[r][c], s[r][c], sp[r][c], spp[r][c]);
            p[r][c] = sp[r][c] * tt[r][c];
        }
    store_tT<TE>(S.ST, f0, e0, s);
    store_tT<TE>(S.PT, f0, e0, p);
}

// Segmented row sums of X[e][f] into acc[row][f] (rows are contiguous runs
// of the tile's pairs; pairs past the end have row -1). Warp w sums pairs
// [w TE/8, (w + 1) TE/8) segment by segment, lane f feature f; a segment that
// starts and ends inside the warp's range is a whole row and is stored
// directly, the range's first and last segments go to two slots. Threads < F
// then merge the slots in pair order, the open row carried across tiles in
// cur/run. Every row's sum is fixed by the tile boundaries (deterministic).
// All threads take part (one barrier inside); a barrier after the call must
// come before the slots, X or the rows are written again.
template <int F, int TE, int K>
__device__ __forceinline__ void row_sums(EdgeSmem<F, K>& S, const float* X, int& cur, float& run) {
    static_assert(F == 32, "lane = feature");
    constexpr int NW = kT / 32, EW = TE / NW;
    const int w = threadIdx.x >> 5, f = threadIdx.x & 31;
    int r0 = -1, nseg = 0;
    float sum = 0.f;
    int row_first = -1, row_last = -1;
    float v_first = 0.f, v_last = 0.f;
    for (int e = w * EW; e < (w + 1) * EW; ++e) {
        const int r = S.row[e];
        if (r < 0) break;
        if (r != r0) {
            if (r0 >= 0) {
                if (nseg == 0) {
                    row_first = r0;
                    v_first = sum;
                } else {
                    S.acc[r0 * F + f] = sum;
                }
                ++nseg;
            }
            r0 = r;
            sum = 0.f;
        }
        sum += X[e * (F + 4) + f];
    }
    if (r0 >= 0) {
        if (nseg == 0) {
            row_first = r0;
            v_first = sum;
        } else {
            row_last = r0;
            v_last = sum;
        }
    }
    S.slot[w][0][f] = v_first;
    S.slot[w][1][f] = v_last;
    if (f == 0) {
        S.slot_row[w][0] = row_first;
        S.slot_row[w][1] = row_last;
    }
    __syncthreads();
    if (threadIdx.x < F) {
#pragma unroll
        for (int k = 0; k < 2 * NW; ++k) {
            const int r = S.slot_row[k >> 1][k & 1];
            if (r < 0) continue;
            const float v = S.slot[k >> 1][k & 1][f];
            if (r == cur) {
                run += v;
            } else {
                if (cur >= 0) S.acc[cur * F + f] = run;
                cur = r;
                run = v;
            }
        }
    }
}

// ------------------------------------------------------------ tangent edge pass: m'
template <int F, int K>
__global__ void __launch_bounds__(kT) k_fm_tangent(PotArgs a, const float* __restrict__ g, float* __restrict__ mdot) {
    using G = Geo<F, K>;
    constexpr int TE = G::TE, FG = G::FG, PS = F + 4;
    extern __shared__ float4 sm4[];
    EdgeSmem<F, K>& S = *reinterpret_cast<EdgeSmem<F, K>*>(sm4);
    const int tid = threadIdx.x, A = a.atoms_per_cta;
    const int a0 = blockIdx.x * A, a1 = min(a.n_atoms, a0 + A), nA = a1 - a0;
    if (nA <= 0) return;
    load_weights(S, a);
    for (int t = tid; t < A * F; t += kT) S.acc[t] = 0.f;
    const long long e_beg = min((long long)a.row_ptr[a0], a.e_cap), e_end = min((long long)a.row_ptr[a1], a.e_cap);
    const int fg = tid % FG, eg = tid / FG, f0 = 4 * fg, e0 = 4 * eg;
    int cur = -1;
    float run = 0.f;
    __syncthreads();
    for (long long t0 = e_beg; t0 < e_end; t0 += TE) {
        edge_setup(S, a, g, t0, e_end, a0);
        __syncthreads();
        float sp[4][4], spp[4][4], tt[4][4];
        filter_hidden(S, e0, f0, sp, spp, tt);
        __syncthreads();
        float phi[4][4], q[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) { phi[r][c] = S.b2[f0 + c]; q[r][c] = 0.f; }
        tgemm<F, TE, F>(S.ST, S.W2, e0, f0, phi);
        tgemm<F, TE, F>(S.PT, S.W2, e0, f0, q);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = e0 + r;
            float dl = S.delta[e], fc = S.fc[e], dfc = S.dfc[e];
            const float* uj = a.u + (size_t)S.j[e] * F + f0;
            float4 o;
            o.x = dl * (dfc * phi[r][0] + fc * q[r][0]) * uj[0];
            o.y = dl * (dfc * phi[r][1] + fc * q[r][1]) * uj[1];
            o.z = dl * (dfc * phi[r][2] + fc * q[r][2]) * uj[2];
            o.w = dl * (dfc * phi[r][3] + fc * q[r][3]) * uj[3];
            *reinterpret_cast<float4*>(S.X + e * PS + f0) = o;
        }
        __syncthreads();
        row_sums<F, TE, K>(S, S.X, cur, run);
        __syncthreads();
    }
    if (tid < F && cur >= 0) S.acc[cur * F + tid] = run;
    __syncthreads();
    for (int t = tid; t < nA * F; t += kT) mdot[(size_t)a0 * F + t] = S.acc[t];
}

// ------------------------------------------------------------ per-atom adjoint pass
// Warp per atom, lane = feature (F = 32). Gradient slots (floats) of the
// per-CTA partial vector: the flat parameter layout (only the blocks this
// pass touches are written).


// out[lane] = sum_k v[k] W[k][lane] (gemv_s) and sum_k v[k] W[lane][k]
// (gemv_t_s, W with row stride 33), the vector in shared memory (one copy
// per warp) read four entries per broadcast load, the sums over k in order.
__device__ __forceinline__ float gemv_s(const float* v, const float* W) {
    const int lane = threadIdx.x & 31;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 32; k += 4) {
        const float4 x = *reinterpret_cast<const float4*>(v + k);
        acc += x.x * W[k * 32 + lane];
        acc += x.y * W[(k + 1) * 32 + lane];
        acc += x.z * W[(k + 2) * 32 + lane];
        acc += x.w * W[(k + 3) * 32 + lane];
    }
    return acc;
}
__device__ __forceinline__ float gemv_t_s(const float* v, const float* W) {
    const int lane = threadIdx.x & 31;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 32; k += 4) {
        const float4 x = *reinterpret_cast<const float4*>(v + k);
        acc += x.x * W[lane * 33 + k];
        acc += x.y * W[lane * 33 + k + 1];
        acc += x.z * W[lane * 33 + k + 2];
        acc += x.w * W[lane * 33 + k + 3];
    }
    return acc;
}
// g[k] += a[k] sa + b[k] sb (a, b in shared memory, one copy per warp)
__device__ __forceinline__ void outer(float* g, const float* a, float sa, const float* b, float sb) {
#pragma unroll
    for (int k = 0; k < 32; k += 4) {
        const float4 x = *reinterpret_cast<const float4*>(a + k), y = *reinterpret_cast<const float4*>(b + k);
        g[k] += x.x * sa + y.x * sb;
        g[k + 1] += x.y * sa + y.y * sb;
        g[k + 2] += x.z * sa + y.z * sb;
        g[k + 3] += x.w * sa + y.w * sb;
    }
}

constexpr int kAtomWarps = 8;

__global__ void __launch_bounds__(kAtomWarps * 32) k_fm_atom(PotArgs a, const float* __restrict__ m,
                                                              const float* __restrict__ mdot,
                                                              float* __restrict__ mbar_psi,
                                                              float* __restrict__ mdotbar_psi,
                                                              float* __restrict__ partial, int n_params,
                                                              const double* __restrict__ c_energy) {
    constexpr int F = 32;
    // U1, U2, R1 as W[k][f] (for x W), then padded copies U1T, U2T, R1T (for
    // x W^T); at the end the same array holds the block's gradient sums
    __shared__ float smw[3 * F * F + 3 * F * 33];
    __shared__ __align__(16) float vbuf[kAtomWarps][12][F];
    float* const U1 = smw;
    float* const U2 = U1 + F * F;
    float* const R1 = U2 + F * F;
    float* const U1T = R1 + F * F;
    float* const U2T = U1T + F * 33;
    float* const R1T = U2T + F * 33;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const float* P = a.P;
    for (int t = tid; t < F * F; t += blockDim.x) {
        int r = t / F, c = t % F;
        float u1 = P[a.off.U1[0] + t], u2 = P[a.off.U2[0] + t], r1 = P[a.off.R1 + t];
        U1[t] = u1; U2[t] = u2; R1[t] = r1;
        U1T[r * 33 + c] = u1; U2T[r * 33 + c] = u2; R1T[r * 33 + c] = r1;
    }
    __syncthreads();
    const float c1 = P[a.off.c1[0] + lane], d1 = P[a.off.d1 + lane], r2 = P[a.off.R2 + lane];
    const float ce = c_energy ? (float)*c_energy : 0.f;        // dL/dE of this frame (energy term)
    float n_here = 0.f, n_sp_here = 0.f;                       // atoms of this warp; of species `lane`
    // per-lane gradient accumulators: column `lane` of dR1, dU2, dU1 (k = 0..31), and vectors
    float gR1[F], gU2[F], gU1[F];
#pragma unroll
    for (int k = 0; k < F; ++k) { gR1[k] = 0.f; gU2[k] = 0.f; gU1[k] = 0.f; }
    float gR2 = 0.f, gd1 = 0.f, gc2 = 0.f, gc1 = 0.f;
    const int S_species = a.off.W_in[0] - a.off.A;   // S * F entries of A
    float gA[16];
#pragma unroll
    for (int z = 0; z < 16; ++z) gA[z] = 0.f;
    const int n_sp = S_species / F;
    // per-warp vectors (one feature per lane) that the matrix-vector products
    // read as broadcasts, four features per load; each slot is written once
    // per atom
    float* const vs = vbuf[w][0];
    auto slot = [&](int k) { return vs + k * F; };
    for (int i = blockIdx.x * kAtomWarps + w; i < a.n_atoms; i += gridDim.x * kAtomWarps) {
        const size_t o = (size_t)i * F + lane;
        const float mv = m[o], md = mdot[o], h1 = a.h[o];
        __syncwarp();                              // the previous atom's slots have been read
        slot(0)[lane] = mv;
        slot(1)[lane] = md;
        slot(2)[lane] = h1;
        __syncwarp();
        const float z = gemv_s(slot(0), U1) + c1;
        const float zd = gemv_s(slot(1), U1);
        const float q = gemv_s(slot(2), R1) + d1;
        float sz, s1z, s2z;
        silu3(z, sz, s1z, s2z);
        const float yd = s1z * zd;                 // tangent of SiLU(z)
        slot(3)[lane] = yd;
        slot(4)[lane] = sz;
        __syncwarp();
        const float h1d = gemv_s(slot(3), U2);     // tangent of h1
        slot(5)[lane] = h1d;
        __syncwarp();
        const float qd = gemv_s(slot(5), R1);
        float sq, s1q, s2q;
        silu3(q, sq, s1q, s2q);
        const float qdb = s1q * r2;                // dPsi/dq'
        const float qb = s2q * qd * r2 - ce * s1q * r2;   // dPsi/dq, with the energy term's seed
        gR2 += s1q * qd - ce * sq;
        gd1 += qb;
        outer(gR1, slot(2), qb, slot(5), qdb);
        slot(6)[lane] = qb;
        slot(7)[lane] = qdb;
        __syncwarp();
        const float hb = gemv_t_s(slot(6), R1T);   // dPsi/dh1
        const float hdb = gemv_t_s(slot(7), R1T);  // dPsi/dh1'
        gc2 += hb;
        outer(gU2, slot(4), hb, slot(3), hdb);
        slot(8)[lane] = hb;
        slot(9)[lane] = hdb;
        __syncwarp();
        const float yb = gemv_t_s(slot(8), U2T);
        const float ydb = gemv_t_s(slot(9), U2T);
        const float zb = yb * s1z + ydb * s2z * zd;
        const float zdb = ydb * s1z;
        gc1 += zb;
        outer(gU1, slot(0), zb, slot(1), zdb);
        slot(10)[lane] = zb;
        slot(11)[lane] = zdb;
        __syncwarp();
        mbar_psi[o] = gemv_t_s(slot(10), U1T);
        mdotbar_psi[o] = gemv_t_s(slot(11), U1T);
        const int sp = a.species[i];
#pragma unroll
        for (int zz = 0; zz < 16; ++zz)
            if (zz == sp) gA[zz] += hb;               // residual h1 = h0 + ... with h0 = A[Z]
        n_here += 1.f;
        if (lane == sp) n_sp_here += 1.f;
    }
    // the block's partials: the warps' sums added in warp order in shared
    // memory, then one row partial[blockIdx * n_params + param]
    __syncthreads();                                   // the weight copies are no longer read
    float* sacc = smw;                                 // 3 F^2 + 4 F + 16 F + 17 floats fit in smw
    float* sR1 = sacc, *sU2 = sR1 + F * F, *sU1 = sU2 + F * F, *sv = sU1 + F * F;   // sv: R2 d1 c2 c1
    float* sA = sv + 4 * F, *sE = sA + 16 * F;                                          // sE: d2, e0[16]
    for (int ww = 0; ww < kAtomWarps; ++ww) {
        if (w == ww) {
            auto put = [&](float* dst, float v) { *dst = ww == 0 ? v : *dst + v; };
#pragma unroll
            for (int k = 0; k < F; ++k) {
                put(sR1 + k * F + lane, gR1[k]);
                put(sU2 + k * F + lane, gU2[k]);
                put(sU1 + k * F + lane, gU1[k]);
            }
            put(sv + lane, gR2);
            put(sv + F + lane, gd1);
            put(sv + 2 * F + lane, gc2);
            put(sv + 3 * F + lane, gc1);
            for (int zz = 0; zz < n_sp && zz < 16; ++zz) put(sA + zz * F + lane, gA[zz]);
            // every atom adds d2 and e0[Z_i] to the energy once (exact counts in FP32)
            if (lane == 0) put(sE, -ce * n_here);
            if (lane < n_sp) put(sE + 1 + lane, -ce * n_sp_here);
        }
        __syncthreads();
    }
    float* out = partial + (size_t)blockIdx.x * n_params;
    for (int t = tid; t < F * F; t += blockDim.x) {
        out[a.off.R1 + t] = sR1[t];
        out[a.off.U2[0] + t] = sU2[t];
        out[a.off.U1[0] + t] = sU1[t];
    }
    for (int t = tid; t < F; t += blockDim.x) {
        out[a.off.R2 + t] = sv[t];
        out[a.off.d1 + t] = sv[F + t];
        out[a.off.c2[0] + t] = sv[2 * F + t];
        out[a.off.c1[0] + t] = sv[3 * F + t];
    }
    for (int t = tid; t < n_sp * F; t += blockDim.x) out[a.off.A + t] = sA[t];
    if (tid == 0) out[a.off.d2] = sE[0];
    if (tid < n_sp) out[a.off.e0 + tid] = sE[1 + tid];
}

// ------------------------------------------------------------ filter-weight gradient edge pass
// Per directed edge (i, j): wbar = Mbar_i * u_j, wdbar = Mdbar_i * u_j (dPsi/dm,
// dPsi/dm' of the receiver), phibar = fc wbar + delta fc' wdbar,
// gbar = delta fc wdbar (adjoint of (SiLU'(a) T) W2),
//   dW2 += SiLU(a)^T phibar + (SiLU'(a) T)^T gbar,  db2 += phibar,
//   abar = (phibar W2^T) SiLU'(a) + (gbar W2^T) T SiLU''(a),  tbar = (gbar W2^T) SiLU'(a),
//   dW1 += e^T abar + e'^T tbar,  db1 += abar;
// and ubar_i = sum_j w_ij * Mbar_j + w'_ij * Mdbar_j (row gather, w symmetric).
template <int F, int K>
__global__ void __launch_bounds__(kT) k_fm_grad_edge(PotArgs a, const float* __restrict__ g,
                                                      const float* __restrict__ mb, const float* __restrict__ mdb,
                                                      float* __restrict__ ubar, float* __restrict__ partial,
                                                      int n_params) {
    using G = Geo<F, K>;
    constexpr int TE = G::TE, FG = G::FG, PS = F + 4;
    extern __shared__ float4 sm4[];
    EdgeSmem<F, K>& S = *reinterpret_cast<EdgeSmem<F, K>*>(sm4);
    const int tid = threadIdx.x, A = a.atoms_per_cta;
    const int a0 = blockIdx.x * A, a1 = min(a.n_atoms, a0 + A), nA = a1 - a0;
    float* out = partial + (size_t)blockIdx.x * n_params;
    // gradient accumulators of this thread: dW2 entries (k, f) = (tid / (F/4)) .. and W1, biases
    constexpr int NW2 = F * F / kT;      // dW2 entries per thread
    float gW2[NW2 > 0 ? NW2 : 1];
#pragma unroll
    for (int q = 0; q < NW2; ++q) gW2[q] = 0.f;
    constexpr int NW1 = (K * F + kT - 1) / kT;   // dW1 entries per thread
    float gW1[NW1];
#pragma unroll
    for (int q = 0; q < NW1; ++q) gW1[q] = 0.f;
    float gb = 0.f;                      // one bias entry (db2: tid < F, db1: the last F threads)
    if (nA > 0) {
        load_weights(S, a);
        for (int t = tid; t < A * F; t += kT) S.acc[t] = 0.f;
    }
    const long long e_beg = nA > 0 ? min((long long)a.row_ptr[a0], a.e_cap) : 0;
    const long long e_end = nA > 0 ? min((long long)a.row_ptr[a1], a.e_cap) : 0;
    const int fg = tid % FG, eg = tid / FG, f0 = 4 * fg, e0 = 4 * eg;
    int cur = -1;
    float run = 0.f;
    __syncthreads();
    for (long long t0 = e_beg; t0 < e_end; t0 += TE) {
        edge_setup(S, a, g, t0, e_end, a0);
        __syncthreads();
        float sp[4][4], spp[4][4], tt[4][4];
        filter_hidden(S, e0, f0, sp, spp, tt);
        __syncthreads();
        float phi[4][4], q[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) { phi[r][c] = S.b2[f0 + c]; q[r][c] = 0.f; }
        tgemm<F, TE, F>(S.ST, S.W2, e0, f0, phi);
        tgemm<F, TE, F>(S.PT, S.W2, e0, f0, q);
        // edge adjoints phibar, gbar (rows of X, Y) and the ubar message (into X after use)
        float phb[4][4], gb4[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = e0 + r;
            int row = S.row[e];
            int i = row < 0 ? a0 : a0 + row;
            float dl = S.delta[e], fc = S.fc[e], dfc = S.dfc[e];
            const float* uj = a.u + (size_t)S.j[e] * F + f0;
            const float* mbi = mb + (size_t)i * F + f0;
            const float* mdbi = mdb + (size_t)i * F + f0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float wb = mbi[c] * uj[c], wdb = mdbi[c] * uj[c];
                phb[r][c] = fc * wb + dl * dfc * wdb;
                gb4[r][c] = dl * fc * wdb;
            }
            *reinterpret_cast<float4*>(S.X + e * PS + f0) = make_float4(phb[r][0], phb[r][1], phb[r][2], phb[r][3]);
            *reinterpret_cast<float4*>(S.Y + e * PS + f0) = make_float4(gb4[r][0], gb4[r][1], gb4[r][2], gb4[r][3]);
        }
        __syncthreads();
        // abar, tbar: need phibar W2^T and gbar W2^T (rows of X, Y as A operand, transposed access)
        float sb[4][4], pb[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) { sb[r][c] = 0.f; pb[r][c] = 0.f; }
        for (int k = 0; k < F; ++k) {
            float4 wv = *reinterpret_cast<const float4*>(S.W2T + k * F + f0);   // W2[f0..f0+3][k]
            float wf[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float xph = S.X[(e0 + r) * PS + k], xg = S.Y[(e0 + r) * PS + k];
#pragma unroll
                for (int c = 0; c < 4; ++c) { sb[r][c] += xph * wf[c]; pb[r][c] += xg * wf[c]; }
            }
        }
        float ab[4][4], tb[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                ab[r][c] = sb[r][c] * sp[r][c] + pb[r][c] * tt[r][c] * spp[r][c];
                tb[r][c] = pb[r][c] * sp[r][c];
            }
        // weight gradients of this tile: dW2 (ST, PT against X, Y), db2; then dW1 (BT, DT against abar, tbar), db1
#pragma unroll
        for (int qq = 0; qq < NW2; ++qq) {
            int idx = tid + qq * kT;
            int k = idx / F, f = idx % F;
            float s = 0.f;
            for (int e = 0; e < TE; ++e) s += S.ST[k * TE + e] * S.X[e * PS + f] + S.PT[k * TE + e] * S.Y[e * PS + f];
            gW2[qq] += s;
        }
        if (tid < F) {
            float s = 0.f;
            for (int e = 0; e < TE; ++e) s += S.X[e * PS + tid];
            gb += s;                                          // db2
        }
        __syncthreads();
        // abar -> X, tbar -> Y (rows)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = e0 + r;
            *reinterpret_cast<float4*>(S.X + e * PS + f0) = make_float4(ab[r][0], ab[r][1], ab[r][2], ab[r][3]);
            *reinterpret_cast<float4*>(S.Y + e * PS + f0) = make_float4(tb[r][0], tb[r][1], tb[r][2], tb[r][3]);
        }
        __syncthreads();
#pragma unroll
        for (int qq = 0; qq < NW1; ++qq) {
            int idx = tid + qq * kT;
            if (idx < K * F) {
                int k = idx / F, f = idx % F;
                float s = 0.f;
                for (int e = 0; e < TE; ++e)
                    s += S.BT[k * TE + e] * S.X[e * PS + f] + S.DT[k * TE + e] * S.Y[e * PS + f];
                gW1[qq] += s;
            }
        }
        if (tid >= kT - F) {
            int f = tid - (kT - F);
            float s = 0.f;
            for (int e = 0; e < TE; ++e) s += S.X[e * PS + f];
            gb += s;                                          // db1 (threads kT-F .. kT-1)
        }
        __syncthreads();
        // ubar message: w * Mbar_j + w' * Mdbar_j with w = fc phi, w' = delta (fc' phi + fc q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = e0 + r;
            float dl = S.delta[e], fc = S.fc[e], dfc = S.dfc[e];
            const float* mbj = mb + (size_t)S.j[e] * F + f0;
            const float* mdbj = mdb + (size_t)S.j[e] * F + f0;
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) o[c] = fc * phi[r][c] * mbj[c] + dl * (dfc * phi[r][c] + fc * q[r][c]) * mdbj[c];
            *reinterpret_cast<float4*>(S.X + e * PS + f0) = make_float4(o[0], o[1], o[2], o[3]);
        }
        __syncthreads();
        row_sums<F, TE, K>(S, S.X, cur, run);
        __syncthreads();
    }
    if (nA > 0) {
        if (tid < F && cur >= 0) S.acc[cur * F + tid] = run;
        __syncthreads();
        for (int t = tid; t < nA * F; t += kT) ubar[(size_t)a0 * F + t] = S.acc[t];
    }
    // CTA partials of the filter weights
#pragma unroll
    for (int qq = 0; qq < NW2; ++qq) out[a.off.W2[0] + tid + qq * kT] = gW2[qq];
#pragma unroll
    for (int qq = 0; qq < NW1; ++qq)
        if (tid + qq * kT < K * F) out[a.off.W1[0] + tid + qq * kT] = gW1[qq];
    if (tid < F) out[a.off.b2[0] + tid] = gb;
    if (tid >= kT - F) out[a.off.b1[0] + tid - (kT - F)] = gb;
}

// ------------------------------------------------------------ tensor-core edge passes (BF16 mode)
// The BF16 weight operands from the FP32 weights in shared memory.
template <int F, int K>
__device__ __forceinline__ void build_tc_weights(const EdgeSmem<F, K>& S, TcWeights<F>& W) {
    for (int t = threadIdx.x; t < F * kKb; t += kT) {
        const int n = t / kKb, k = t % kKb;
        *reinterpret_cast<__nv_bfloat16*>(W.w1t + tile_offset(n, k, kKb)) =
            __float2bfloat16_rn(k < K ? S.W1[k * F + n] : 0.f);
    }
    for (int t = threadIdx.x; t < F * F; t += kT) {
        const int n = t / F, k = t % F;
        *reinterpret_cast<__nv_bfloat16*>(W.w2t + tile_offset(n, k, F)) = __float2bfloat16_rn(S.W2[k * F + n]);
        *reinterpret_cast<__nv_bfloat16*>(W.w2n + tile_offset(n, k, F)) = __float2bfloat16_rn(S.W2[n * F + k]);
    }
}

// Two 32-column FP32 accumulators of the tile (tensor-memory columns t ..
// t + 31 and t + 32 .. t + 63, lane = pair) into rows d0[e][.], d1[e][.]
// (stride F + 4): warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31 of the
// accumulator w / 4.
template <int F>
__device__ __forceinline__ void tmem_rows(uint32_t t, float* d0, float* d1) {
    static_assert(F == 32 && kT == 256, "eight warps, one 32-column half each");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = w & 3, h = w >> 2;
    const uint32_t ta = t + ((uint32_t)(32 * qd) << 16) + (uint32_t)(32 * h);
    float v[32];
    tmem_ld16x2(ta, v, ta + 16, v + 16);
    float* dst = (h ? d1 : d0) + (32 * qd + lane) * (F + 4);
#pragma unroll
    for (int c = 0; c < 32; c += 4) *reinterpret_cast<float4*>(dst + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
}

// Bounded completion waits on the CTA's MMA barrier (all threads): the
// parity of the oldest commit not yet waited for; a wait that gives up clears
// ok and records its parity, so that the MMAs in flight can be drained
// before the tensor memory is freed.
struct MmaWaits {
    uint32_t phase = 0, fail_phase = 0;
    bool ok = true, failed = false;
    __device__ __forceinline__ void wait(uint64_t* mbar) {
        const bool done = mbar_wait(mbar, phase, kFmWait);
        if (!done && !failed) {
            failed = true;
            fail_phase = phase;
        }
        ok = ok && done;
        phase ^= 1;
        fence_after_sync();
    }
    // end of the kernel: drain, then bit 0 (a wait gave up) and bit 1 (its MMAs did not drain) of *status
    __device__ __forceinline__ void finish(uint64_t* mbar, uint32_t taddr, uint32_t ncols, int* status) {
        const bool drained = !failed || mbar_wait(mbar, fail_phase, kFmWait);
        fence_before_sync();
        ok = __syncthreads_and(ok);
        if (threadIdx.x < 32) tmem_dealloc(taddr, ncols);
        if (!ok && threadIdx.x == 0) atomicOr(status, drained ? 1 : 3);
    }
};

// Barrier that also makes the operands written by this CTA's threads visible
// to the tensor cores; returns the AND of ok over the CTA.
__device__ __forceinline__ bool operands_ready(bool ok) {
    fence_proxy_async();
    fence_before_sync();
    ok = __syncthreads_and(ok);
    fence_after_sync();
    return ok;
}

// m' by the tensor cores (k_fm_tangent with MMA1 and MMA2; see above).
template <int F, int K>
__global__ void __launch_bounds__(kT) k_fm_tangent_tc(PotArgs a, const float* __restrict__ g, float* __restrict__ mdot,
                                                       int* status) {
    using G = Geo<F, K>;
    constexpr int TE = G::TE, FG = G::FG, PS = F + 4;
    static_assert(TE == 128 && F == 32, "one pair per tensor-memory lane");
    extern __shared__ float4 sm4[];
    TangTc<F, K>& T = *reinterpret_cast<TangTc<F, K>*>(sm4);
    EdgeSmem<F, K>& S = T.e;
    unsigned char* const a2 = reinterpret_cast<unsigned char*>(S.ST);   // SiLU(a) | SiLU'(a) T, 16 KB
    unsigned char* const a1 = reinterpret_cast<unsigned char*>(S.PT);   // e | e', 8 KB
    const int tid = threadIdx.x, A = a.atoms_per_cta;
    const int a0 = blockIdx.x * A, a1_ = min(a.n_atoms, a0 + A), nA = a1_ - a0;
    if (nA <= 0) return;
    load_weights(S, a);
    for (int t = tid; t < A * F; t += kT) S.acc[t] = 0.f;
    __syncthreads();
    build_tc_weights(S, T.w);
    if (tid == 0) mbar_init(&T.mbar, 1);
    if (tid < 32) tmem_alloc(&T.taddr, 64);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tXY = T.taddr, idesc = idesc_bf16_f32(128, F);
    const uint32_t sA1 = smem_u32(a1), sA2 = smem_u32(a2);
    const uint32_t sW1 = smem_u32(T.w.w1t), sW2 = smem_u32(T.w.w2t);
    MmaWaits mw;
    const long long e_beg = min((long long)a.row_ptr[a0], a.e_cap), e_end = min((long long)a.row_ptr[a1_], a.e_cap);
    const int fg = tid % FG, eg = tid / FG, f0 = 4 * fg, e0 = 4 * eg;
    int cur = -1;
    float run = 0.f;
    PairIn nx;                                           // the next tile's pair inputs (threads < TE)
    if (tid < TE) {
        pair_idx(a, e_beg + tid, e_end, nx);
        pair_pos(a, g, nx);
    }
    for (long long t0 = e_beg; t0 < e_end; t0 += TE) {
        if (tid < TE) {
            edge_setup_in(S, a, nx, a0, a1);
            pair_idx(a, t0 + TE + tid, e_end, nx);       // in flight during this tile
        }
        mw.ok = operands_ready(mw.ok);
        if (mw.ok) {
            if (tid == 0) {
                mma_bf16(tXY, make_desc(sA1, 128, kKb * 16), make_desc(sW1, 128, kKb * 16), idesc, 0);
                mma_bf16(tXY + F, make_desc(sA1 + TE * kKb * 2, 128, kKb * 16), make_desc(sW1, 128, kKb * 16), idesc, 0);
                mma_commit(&T.mbar);
            }
            mw.wait(&T.mbar);
        }
        tmem_rows<F>(tXY, S.X, S.Y);                     // a - b1 | T
        if (tid < TE) pair_pos(a, g, nx);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float sv[4], pv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float sp, spp;
                silu3(S.X[(e0 + r) * PS + f0 + c] + S.b1[f0 + c], sv[c], sp, spp);
                pv[c] = sp * S.Y[(e0 + r) * PS + f0 + c];
            }
            st_k4(a2, e0 + r, f0, F, sv[0], sv[1], sv[2], sv[3]);
            st_k4(a2 + TE * F * 2, e0 + r, f0, F, pv[0], pv[1], pv[2], pv[3]);
        }
        mw.ok = operands_ready(mw.ok);
        if (mw.ok) {
            if (tid == 0) {
#pragma unroll
                for (int kk = 0; kk < F / 16; ++kk) {
                    mma_bf16(tXY, make_desc(sA2 + kk * 256, 128, F * 16), make_desc(sW2 + kk * 256, 128, F * 16), idesc,
                             kk > 0);
                    mma_bf16(tXY + F, make_desc(sA2 + TE * F * 2 + kk * 256, 128, F * 16),
                             make_desc(sW2 + kk * 256, 128, F * 16), idesc, kk > 0);
                }
                mma_commit(&T.mbar);
            }
            mw.wait(&T.mbar);
        }
        tmem_rows<F>(tXY, S.X, S.Y);                     // phi - b2 | q
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {                     // the message over this thread's own block of X
            const int e = e0 + r;
            const float dl = S.delta[e], fc = S.fc[e], dfc = S.dfc[e];
            const float* uj = a.u + (size_t)S.j[e] * F + f0;
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float phi = S.X[e * PS + f0 + c] + S.b2[f0 + c], q = S.Y[e * PS + f0 + c];
                o[c] = dl * (dfc * phi + fc * q) * uj[c];
            }
            *reinterpret_cast<float4*>(S.X + e * PS + f0) = make_float4(o[0], o[1], o[2], o[3]);
        }
        __syncthreads();
        row_sums<F, TE, K>(S, S.X, cur, run);
        __syncthreads();
    }
    if (tid < F && cur >= 0) S.acc[cur * F + tid] = run;
    __syncthreads();
    for (int t = tid; t < nA * F; t += kT) mdot[(size_t)a0 * F + t] = S.acc[t];
    mw.finish(&T.mbar, T.taddr, 64, status);
}

// Filter-weight gradients and ubar by the tensor cores (k_fm_grad_edge with
// MMA1-3 and the weight-gradient products; see above).
template <int F, int K>
__global__ void __launch_bounds__(kT, 1) k_fm_grad_edge_tc(PotArgs a, const float* __restrict__ g,
                                                         const float* __restrict__ mb, const float* __restrict__ mdb,
                                                         float* __restrict__ ubar, float* __restrict__ partial,
                                                         int n_params, int* status) {
    using G = Geo<F, K>;
    constexpr int TE = G::TE, FG = G::FG, PS = F + 4;
    static_assert(TE == 128 && F == 32 && 2 * K <= 64, "tensor-core operand shapes");
    extern __shared__ float4 sm4[];
    GradTc<F, K>& T = *reinterpret_cast<GradTc<F, K>*>(sm4);
    EdgeSmem<F, K>& S = T.e;
    unsigned char* const opA = reinterpret_cast<unsigned char*>(S.ST);   // weight-gradient A operand (ST and PT)
    const int tid = threadIdx.x, A = a.atoms_per_cta;
    const int a0 = blockIdx.x * A, a1 = min(a.n_atoms, a0 + A), nA = a1 - a0;
    float* out = partial + (size_t)blockIdx.x * n_params;
    if (nA > 0) {
        load_weights(S, a);
        for (int t = tid; t < A * F; t += kT) S.acc[t] = 0.f;
    }
    __syncthreads();
    if (nA > 0) build_tc_weights(S, T.w);
    if (tid == 0) mbar_init(&T.mbar, 1);
    if (tid < 32) tmem_alloc(&T.taddr, 256);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    // tensor memory: MMA1-3 results in columns [0, 64), D1 in [64, 128), D2 in [128, 192)
    const uint32_t tXY = T.taddr, tD1 = tXY + 64, tD2 = tXY + 128;
    const uint32_t idesc = idesc_bf16_f32(128, F), idesc_w = idesc_bf16_f32(128, 64);
    const uint32_t sA1 = smem_u32(T.a1), sA2 = smem_u32(T.a2), sA3 = smem_u32(T.a3), sB = smem_u32(T.b);
    const uint32_t sOA = smem_u32(opA);
    const uint32_t sW1 = smem_u32(T.w.w1t), sW2T = smem_u32(T.w.w2t), sW2N = smem_u32(T.w.w2n);
    MmaWaits mw;
    bool any = false, pending = false;   // a weight-gradient MMA was issued; the last commit is not yet waited for
    const long long e_beg = nA > 0 ? min((long long)a.row_ptr[a0], a.e_cap) : 0;
    const long long e_end = nA > 0 ? min((long long)a.row_ptr[a1], a.e_cap) : 0;
    const int fg = tid % FG, eg = tid / FG, f0 = 4 * fg, e0 = 4 * eg;
    int cur = -1;
    float run = 0.f;
    PairIn nx;                                           // the next tile's pair inputs (threads < TE)
    if (tid < TE) {
        pair_idx(a, e_beg + tid, e_end, nx);
        pair_pos(a, g, nx);
    }
    for (long long t0 = e_beg; t0 < e_end; t0 += TE) {
        if (tid < TE) {
            edge_setup_in(S, a, nx, a0, &T.a1[0][0]);
            pair_idx(a, t0 + TE + tid, e_end, nx);       // in flight during this tile
        }
        if (pending) {                                   // the previous tile's D2 product reads A and B
            mw.wait(&T.mbar);
            pending = false;
        }
        mw.ok = operands_ready(mw.ok);
        if (mw.ok) {                                     // MMA1: a - b1 | T
            if (tid == 0) {
                mma_bf16(tXY, make_desc(sA1, 128, kKb * 16), make_desc(sW1, 128, kKb * 16), idesc, 0);
                mma_bf16(tXY + F, make_desc(sA1 + TE * kKb * 2, 128, kKb * 16), make_desc(sW1, 128, kKb * 16), idesc, 0);
                mma_commit(&T.mbar);
            }
            mw.wait(&T.mbar);
        }
        tmem_rows<F>(tXY, S.X, S.Y);
        if (tid < TE) pair_pos(a, g, nx);
        __syncthreads();
        float sp[4][4], spp[4][4], tt[4][4];
        {
            float sv[4][4], pv[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    tt[r][c] = S.Y[(e0 + r) * PS + f0 + c];
                    silu3(S.X[(e0 + r) * PS + f0 + c] + S.b1[f0 + c], sv[r][c], sp[r][c], spp[r][c]);
                    pv[r][c] = sp[r][c] * tt[r][c];
                }
                st_k4(&T.a2[0][0], e0 + r, f0, F, sv[r][0], sv[r][1], sv[r][2], sv[r][3]);
                st_k4(&T.a2[1][0], e0 + r, f0, F, pv[r][0], pv[r][1], pv[r][2], pv[r][3]);
            }
            // weight-gradient A rows 0-63: SiLU(a)^T, (SiLU'(a) T)^T (feature rows, pair columns)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                st_k4(opA, f0 + c, e0, TE, sv[0][c], sv[1][c], sv[2][c], sv[3][c]);
                st_k4(opA, F + f0 + c, e0, TE, pv[0][c], pv[1][c], pv[2][c], pv[3][c]);
            }
        }
        // rows 64 ..: e^T, e'^T (K rows each), zero rows, and a row of ones (127: the bias sums)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = tid + kT * i, r = 64 + (c >> 4), k8 = (c & 15) * 8;
            uint4 w = r == 127 ? make_uint4(kBf16Ones, kBf16Ones, kBf16Ones, kBf16Ones) : make_uint4(0u, 0u, 0u, 0u);
            if (r < 64 + 2 * K) {
                const float* src = (r < 64 + K ? S.BT + (r - 64) * TE : S.DT + (r - 64 - K) * TE) + k8;
                const float4 x0 = *reinterpret_cast<const float4*>(src), x1 = *reinterpret_cast<const float4*>(src + 4);
                w = make_uint4(bf16x2(x0.x, x0.y), bf16x2(x0.z, x0.w), bf16x2(x1.x, x1.y), bf16x2(x1.z, x1.w));
            }
            *reinterpret_cast<uint4*>(opA + tile_offset(r, k8, TE)) = w;
        }
        mw.ok = operands_ready(mw.ok);
        if (mw.ok) {                                     // MMA2: phi - b2 | q
            if (tid == 0) {
#pragma unroll
                for (int kk = 0; kk < F / 16; ++kk) {
                    mma_bf16(tXY, make_desc(sA2 + kk * 256, 128, F * 16), make_desc(sW2T + kk * 256, 128, F * 16),
                             idesc, kk > 0);
                    mma_bf16(tXY + F, make_desc(sA2 + TE * F * 2 + kk * 256, 128, F * 16),
                             make_desc(sW2T + kk * 256, 128, F * 16), idesc, kk > 0);
                }
                mma_commit(&T.mbar);
            }
            mw.wait(&T.mbar);
        }
        tmem_rows<F>(tXY, T.Z[0], T.Z[1]);
        __syncthreads();
        float phi[4][4], q[4][4];
        {
            // edge adjoints phibar, gbar: MMA3 A rows, weight-gradient B rows
            float phb[4][4], gb4[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int e = e0 + r;
                const int row = S.row[e];
                const int i = row < 0 ? a0 : a0 + row;
                const float dl = S.delta[e], fc = S.fc[e], dfc = S.dfc[e];
                const float* uj = a.u + (size_t)S.j[e] * F + f0;
                const float* mbi = mb + (size_t)i * F + f0;
                const float* mdbi = mdb + (size_t)i * F + f0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    phi[r][c] = T.Z[0][e * PS + f0 + c] + S.b2[f0 + c];
                    q[r][c] = T.Z[1][e * PS + f0 + c];
                    const float wb = mbi[c] * uj[c], wdb = mdbi[c] * uj[c];
                    phb[r][c] = fc * wb + dl * dfc * wdb;
                    gb4[r][c] = dl * fc * wdb;
                }
                st_k4(&T.a3[0][0], e, f0, F, phb[r][0], phb[r][1], phb[r][2], phb[r][3]);
                st_k4(&T.a3[1][0], e, f0, F, gb4[r][0], gb4[r][1], gb4[r][2], gb4[r][3]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {                // B1 rows f (phibar) and F + f (gbar), pair columns e0 ..
                st_k4(T.b, f0 + c, e0, TE, phb[0][c], phb[1][c], phb[2][c], phb[3][c]);
                st_k4(T.b, F + f0 + c, e0, TE, gb4[0][c], gb4[1][c], gb4[2][c], gb4[3][c]);
            }
        }
        mw.ok = operands_ready(mw.ok);
        if (mw.ok) {                                     // D1 += A B1^T; MMA3: sb | pb
            if (tid == 0) {
#pragma unroll
                for (int kk = 0; kk < TE / 16; ++kk)
                    mma_bf16(tD1, make_desc(sOA + kk * 256, 128, TE * 16), make_desc(sB + kk * 256, 128, TE * 16),
                             idesc_w, any || kk > 0);
#pragma unroll
                for (int kk = 0; kk < F / 16; ++kk) {
                    mma_bf16(tXY, make_desc(sA3 + kk * 256, 128, F * 16), make_desc(sW2N + kk * 256, 128, F * 16),
                             idesc, kk > 0);
                    mma_bf16(tXY + F, make_desc(sA3 + TE * F * 2 + kk * 256, 128, F * 16),
                             make_desc(sW2N + kk * 256, 128, F * 16), idesc, kk > 0);
                }
                mma_commit(&T.mbar);
            }
        }
        if (mw.ok) mw.wait(&T.mbar);
        tmem_rows<F>(tXY, T.Z[0], T.Z[1]);
        __syncthreads();
        float ab[4][4], tb[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float sb = T.Z[0][(e0 + r) * PS + f0 + c], pb = T.Z[1][(e0 + r) * PS + f0 + c];
                ab[r][c] = sb * sp[r][c] + pb * tt[r][c] * spp[r][c];
                tb[r][c] = pb * sp[r][c];
            }
        // B2 = [abar | tbar] over B1, which the completed D1 product read
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            st_k4(T.b, f0 + c, e0, TE, ab[0][c], ab[1][c], ab[2][c], ab[3][c]);
            st_k4(T.b, F + f0 + c, e0, TE, tb[0][c], tb[1][c], tb[2][c], tb[3][c]);
        }
        mw.ok = operands_ready(mw.ok);
        if (mw.ok) {                                     // D2 += A B2^T
            if (tid == 0) {
#pragma unroll
                for (int kk = 0; kk < TE / 16; ++kk)
                    mma_bf16(tD2, make_desc(sOA + kk * 256, 128, TE * 16), make_desc(sB + kk * 256, 128, TE * 16),
                             idesc_w, any || kk > 0);
                mma_commit(&T.mbar);
            }
            pending = true;
            any = true;
        }
        // ubar message: w * Mbar_j + w' * Mdbar_j with w = fc phi, w' = delta (fc' phi + fc q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = e0 + r;
            const float dl = S.delta[e], fc = S.fc[e], dfc = S.dfc[e];
            const float* mbj = mb + (size_t)S.j[e] * F + f0;
            const float* mdbj = mdb + (size_t)S.j[e] * F + f0;
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) o[c] = fc * phi[r][c] * mbj[c] + dl * (dfc * phi[r][c] + fc * q[r][c]) * mdbj[c];
            *reinterpret_cast<float4*>(S.X + e * PS + f0) = make_float4(o[0], o[1], o[2], o[3]);
        }
        __syncthreads();
        row_sums<F, TE, K>(S, S.X, cur, run);
        __syncthreads();
    }
    if (nA > 0) {
        if (tid < F && cur >= 0) S.acc[cur * F + tid] = run;
        __syncthreads();
        for (int t = tid; t < nA * F; t += kT) ubar[(size_t)a0 * F + t] = S.acc[t];
    }
    // CTA partials of the filter weights from D1 and D2
    if (pending) mw.wait(&T.mbar);
    const bool ok = __syncthreads_and(mw.ok);
    float* st = S.X;                                     // staging: D1 blocks, D2 blocks, the bias sums
    const int w = tid >> 5, lane = tid & 31;
    if (ok && any && w == 3) {                           // row 127 (lane 31 of warp 3): sum over pairs of phibar, abar
        float v[32];
        const uint32_t ta = tD1 + (96u << 16), tb = tD2 + (96u << 16);
        tmem_ld16x2(ta, v, ta + 16, v + 16);
        if (lane == 31)
#pragma unroll
            for (int f = 0; f < 32; ++f) st[3072 + f] = v[f];
        tmem_ld16x2(tb, v, tb + 16, v + 16);
        if (lane == 31)
#pragma unroll
            for (int f = 0; f < 32; ++f) st[3104 + f] = v[f];
    }
    if (ok && any && w < 3) {
        float v[32];
        if (w < 2) {                                     // lanes 32 w + lane: SiLU(a)^T rows (w 0), (SiLU'(a) T)^T rows (w 1)
            const uint32_t ta = tD1 + ((uint32_t)(32 * w) << 16) + (w == 0 ? 0u : 32u);
            tmem_ld16x2(ta, v, ta + 16, v + 16);
#pragma unroll
            for (int f = 0; f < 32; ++f) st[(w * 32 + lane) * 32 + f] = v[f];
        } else {                                         // lanes 64 + lane: e^T (lane < K), e'^T (K <= lane < 2K)
            const uint32_t ta = tD2 + (64u << 16);       // both column halves (the address is warp-uniform)
            tmem_ld16x2(ta, v, ta + 16, v + 16);
            if (lane < K)
#pragma unroll
                for (int f = 0; f < 32; ++f) st[2048 + lane * 32 + f] = v[f];
            tmem_ld16x2(ta + 32, v, ta + 48, v + 16);
            if (lane >= K && lane < 2 * K)
#pragma unroll
                for (int f = 0; f < 32; ++f) st[2048 + lane * 32 + f] = v[f];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < F * F; idx += kT) out[a.off.W2[0] + idx] = (ok && any) ? st[idx] + st[1024 + idx] : 0.f;
    for (int idx = tid; idx < K * F; idx += kT)
        out[a.off.W1[0] + idx] = (ok && any) ? st[2048 + idx] + st[2048 + K * F + idx] : 0.f;
    if (tid < F) out[a.off.b2[0] + tid] = (ok && any) ? st[3072 + tid] : 0.f;
    if (tid < F) out[a.off.b1[0] + tid] = (ok && any) ? st[3104 + tid] : 0.f;
    mw.finish(&T.mbar, T.taddr, 256, status);
}

// dW_in += h0_i^T ubar_i, dA[Z_i] += ubar_i W_in^T (warp per atom, F = 32)
__global__ void __launch_bounds__(kAtomWarps * 32) k_fm_input(PotArgs a, const float* __restrict__ ubar,
                                                               float* __restrict__ partial, int n_params) {
    constexpr int F = 32;
    __shared__ float WinT[F * 33];     // W_in[k][f] padded, for x W_in^T
    __shared__ __align__(16) float vbuf[kAtomWarps][2][F];   // per-warp h0 and ubar of the atom
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int t = tid; t < F * F; t += blockDim.x) WinT[(t / F) * 33 + t % F] = a.P[a.off.W_in[0] + t];
    __syncthreads();
    float gW[F];
#pragma unroll
    for (int k = 0; k < F; ++k) gW[k] = 0.f;
    float gA[16];
#pragma unroll
    for (int z = 0; z < 16; ++z) gA[z] = 0.f;
    const int n_sp = (a.off.W_in[0] - a.off.A) / F;
    for (int i = blockIdx.x * kAtomWarps + w; i < a.n_atoms; i += gridDim.x * kAtomWarps) {
        const int sp = a.species[i];
        const float ub = ubar[(size_t)i * F + lane];
        const float h0 = a.P[a.off.A + sp * F + lane];
        __syncwarp();                              // the previous atom's vectors have been read
        vbuf[w][0][lane] = h0;
        vbuf[w][1][lane] = ub;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < F; k += 4) {
            const float4 h = *reinterpret_cast<const float4*>(&vbuf[w][0][k]);
            gW[k] += h.x * ub;
            gW[k + 1] += h.y * ub;
            gW[k + 2] += h.z * ub;
            gW[k + 3] += h.w * ub;
        }
        float t = gemv_t_s(vbuf[w][1], WinT);
#pragma unroll
        for (int zz = 0; zz < 16; ++zz)
            if (zz == sp) gA[zz] += t;
    }
    // the warps' sums added in warp order in shared memory, one row per block
    __syncthreads();
    float* sW = WinT;                                  // the W_in gradient: F^2 of its F * 33 floats
    __shared__ float sA[16 * F];
    for (int ww = 0; ww < kAtomWarps; ++ww) {
        if (w == ww) {
#pragma unroll
            for (int k = 0; k < F; ++k) sW[k * F + lane] = ww == 0 ? gW[k] : sW[k * F + lane] + gW[k];
            for (int zz = 0; zz < n_sp && zz < 16; ++zz)
                sA[zz * F + lane] = ww == 0 ? gA[zz] : sA[zz * F + lane] + gA[zz];
        }
        __syncthreads();
    }
    float* out = partial + (size_t)blockIdx.x * n_params;
    for (int t = tid; t < F * F; t += blockDim.x) out[a.off.W_in[0] + t] = sW[t];
    for (int t = tid; t < n_sp * F; t += blockDim.x) out[a.off.A + t] = sA[t];
}

// Energy term of one frame: E = sum over the systems of the model's energies,
// r = (E - E_ref) / N; loss += lambda r^2 / M and c_E = dL/dE = 2 lambda r / (M N).
__global__ void k_fm_energy_term(int n_sys, const double* __restrict__ E, const double* __restrict__ e_ref,
                                 double lambda, int n_atoms, double inv_frames, double* __restrict__ c_energy,
                                 double* __restrict__ loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double e = 0.0;
    for (int k = 0; k < n_sys; ++k) e += E[k];
    const double r = (e - *e_ref) / (double)n_atoms;
    *loss += lambda * r * r * inv_frames;
    *c_energy = 2.0 * lambda * r * inv_frames / (double)n_atoms;
}

// grad[p] -= sum_c partial[c][p] for p in up to four ranges [p0, p1) of
// the parameter vector (one launch): 32 parameters per block, each summed by
// kRedG threads; thread g keeps eight FP64 sums over rows
// c = g + kRedG (8k + u), u = 0..7 (eight loads in flight), adds them
// pairwise in u order, and the kRedG thread sums are added in g order: one
// order for any grid.
constexpr int kRedP = 32, kRedG = 16, kRedU = 8, kRedMax = 4;
struct RedRanges {
    int n = 0;
    int p0[kRedMax] = {}, p1[kRedMax] = {};
    int blk0[kRedMax + 1] = {};          // first block of each range; blk0[n] = the grid
};

__global__ void __launch_bounds__(kRedP * kRedG) k_fm_reduce(const float* __restrict__ partial, int n_rows,
                                                               int n_params, RedRanges rr,
                                                               double* __restrict__ grad) {
    __shared__ double part[kRedG][kRedP];
    int r = 0;
    while (r + 1 < rr.n && (int)blockIdx.x >= rr.blk0[r + 1]) ++r;
    const int lp = threadIdx.x % kRedP, g = threadIdx.x / kRedP;
    const int p = rr.p0[r] + ((int)blockIdx.x - rr.blk0[r]) * kRedP + lp;
    double acc[kRedU];
#pragma unroll
    for (int u = 0; u < kRedU; ++u) acc[u] = 0.0;
    if (p < rr.p1[r]) {
        const float* col = partial + p;
        int c = g;
        for (; c + (kRedU - 1) * kRedG < n_rows; c += kRedU * kRedG) {
#pragma unroll
            for (int u = 0; u < kRedU; ++u) acc[u] += (double)col[(size_t)(c + u * kRedG) * n_params];
        }
#pragma unroll
        for (int u = 0; u < kRedU - 1; ++u)             // the rest: fewer than kRedU rows
            if (c + u * kRedG < n_rows) acc[u] += (double)col[(size_t)(c + u * kRedG) * n_params];
    }
    part[g][lp] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    __syncthreads();
    if (g == 0 && p < rr.p1[r]) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kRedG; ++k) t += part[k][lp];
        grad[p] -= t;
    }
}

// The reduction of the partial rows over the given parameter ranges (one launch).
void fm_reduce(const float* partial, int n_rows, int n_params, std::initializer_list<std::pair<int, int>> ranges,
               double* grad, cudaStream_t s) {
    RedRanges rr;
    int blocks = 0;
    for (const auto& pr : ranges) {
        if (pr.second <= pr.first || rr.n == kRedMax) continue;
        rr.p0[rr.n] = pr.first;
        rr.p1[rr.n] = pr.second;
        rr.blk0[rr.n] = blocks;
        blocks += (pr.second - pr.first + kRedP - 1) / kRedP;
        ++rr.n;
    }
    rr.blk0[rr.n] = blocks;
    if (blocks == 0) return;
    k_fm_reduce<<<blocks, kRedP * kRedG, 0, s>>>(partial, n_rows, n_params, rr, grad);
}

// out += scale * sum v (one block; each thread four interleaved FP64 sums,
// so four loads are in flight, then a fixed-order tree).
constexpr int kSumT = 1024;
__global__ void __launch_bounds__(kSumT) k_sum_all(int n, const double* __restrict__ v, double scale,
                                                   double* __restrict__ out) {
    __shared__ double sh[kSumT];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int i = threadIdx.x;
    for (; i + 3 * kSumT < n; i += 4 * kSumT) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += v[i + u * kSumT];
    }
#pragma unroll
    for (int u = 0; u < 3; ++u)
        if (i + u * kSumT < n) acc[u] += v[i + u * kSumT];
    sh[threadIdx.x] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    __syncthreads();
    for (int w = kSumT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out += scale * sh[0];
}

template <int F, int K>
size_t edge_smem() { return sizeof(EdgeSmem<F, K>); }

template <int F, int K>
void tangent_go(const PotArgs& a, const float* g, float* mdot, cudaStream_t s) {
    smem_opt_in((const void*)k_fm_tangent<F, K>, (int)edge_smem<F, K>());
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    k_fm_tangent<F, K><<<grid, kT, edge_smem<F, K>(), s>>>(a, g, mdot);
}

template <int F, int K>
void tangent_tc_go(const PotArgs& a, const float* g, float* mdot, int* status, cudaStream_t s) {
    smem_opt_in((const void*)k_fm_tangent_tc<F, K>, (int)sizeof(TangTc<F, K>));
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    k_fm_tangent_tc<F, K><<<grid, kT, sizeof(TangTc<F, K>), s>>>(a, g, mdot, status);
}

template <int F, int K>
void grad_edge_tc_go(const PotArgs& a, const float* g, const float* mb, const float* mdb, float* ubar, float* partial,
                     int n_params, int* status, cudaStream_t s) {
    static_assert(sizeof(GradTc<F, K>) <= 227 * 1024, "shared memory of one CTA");
    smem_opt_in((const void*)k_fm_grad_edge_tc<F, K>, (int)sizeof(GradTc<F, K>));
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    k_fm_grad_edge_tc<F, K><<<grid, kT, sizeof(GradTc<F, K>), s>>>(a, g, mb, mdb, ubar, partial, n_params, status);
}

template <int F, int K>
void grad_edge_go(const PotArgs& a, const float* g, const float* mb, const float* mdb, float* ubar, float* partial,
                  int n_params, cudaStream_t s) {
    smem_opt_in((const void*)k_fm_grad_edge<F, K>, (int)edge_smem<F, K>());
    int grid = (a.n_atoms + a.atoms_per_cta - 1) / a.atoms_per_cta;
    k_fm_grad_edge<F, K><<<grid, kT, edge_smem<F, K>(), s>>>(a, g, mb, mdb, ubar, partial, n_params);
}

}  // namespace

bool fm_supported(int F, int K, int L) { return F == 32 && (K == 8 || K == 16) && L == 1; }

namespace {
int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    return sms;
}

// Atoms per CTA of an edge pass that runs `per_sm` CTAs per SM: the atoms
// shared by one wave of CTAs (no partial last wave, fewer ragged tiles), at
// most kFmAtomsMax.
int fm_edge_atoms(int n_atoms, int per_sm) {
    const int ctas = device_sms() * per_sm;
    return std::max(1, std::min(kFmAtomsMax, (n_atoms + ctas - 1) / ctas));
}
}  // namespace

// The gradient edge pass (one CTA per SM, one partial row per CTA).
int fm_edge_ctas(int n_atoms) {
    const int apc = fm_edge_atoms(n_atoms, 1);
    return (n_atoms + apc - 1) / apc;
}

// The per-atom adjoint pass: one block per SM (its registers allow one), one partial row per block.
int fm_atom_ctas(int n_atoms) { return std::max(1, std::min(device_sms(), (n_atoms + kAtomWarps - 1) / kAtomWarps)); }

namespace {
// The input-gradient pass: three blocks per SM, one partial row per block.
int fm_input_ctas(int n_atoms) {
    return std::max(1, std::min(3 * device_sms(), (n_atoms + kAtomWarps - 1) / kAtomWarps));
}
}  // namespace

// Rows of the per-atom passes' partial buffer.
int fm_atom_rows(int n_atoms) { return std::max(fm_atom_ctas(n_atoms), fm_input_ctas(n_atoms)); }

// One frame's contribution: g from the forces already in p.force, then the
// three passes; grad_out accumulates -dPsi/dtheta (+ c_E dE/dtheta with the
// energy term), loss_out the loss. e_ref: this frame's reference energy on
// the device, or null for force matching alone.
void launch_fm_frame(const PotArgs& p, int K, const double* f_ref, double c_loss, float* g, double* sq,
                     const float* m, float* mdot, float* mbar_psi, float* mdotbar_psi, float* ubar, float* partial_e,
                     float* partial_a, int n_params, double* grad, double* loss, const FmEnergy& en,
                     bool tensor_cores, int* status, cudaStream_t s) {
    const int n = p.n_atoms;
    if (n == 0) return;
    k_fm_residual<<<(n + 255) / 256, 256, 0, s>>>(n, p.force, f_ref, c_loss, g, sq);
    k_sum_all<<<1, kSumT, 0, s>>>(n, sq, 0.5 * c_loss, loss);
    if (en.e_ref) {
        k_fm_energy_term<<<1, 32, 0, s>>>(en.n_sys, en.E, en.e_ref, en.lambda, n, en.inv_frames, en.c_energy, loss);
        count_launch();
    }
    PotArgs a = p;
    a.atoms_per_cta = fm_edge_atoms(n, 2);               // the tangent pass: two CTAs per SM
    if (tensor_cores) {
        if (K == 8) tangent_tc_go<32, 8>(a, g, mdot, status, s);
        else tangent_tc_go<32, 16>(a, g, mdot, status, s);
    } else {
        if (K == 8) tangent_go<32, 8>(a, g, mdot, s);
        else tangent_go<32, 16>(a, g, mdot, s);
    }
    // every row of a pass's partials holds every entry of the parameter
    // blocks that pass writes; only those blocks are reduced
    const ModelOffsets& o = a.off;
    const int F = 32, S = (o.W_in[0] - o.A) / F;
    const int ga = fm_atom_ctas(n), ra = ga;             // one partial row per per-atom block
    k_fm_atom<<<ga, kAtomWarps * 32, 0, s>>>(a, m, mdot, mbar_psi, mdotbar_psi, partial_a, n_params,
                                             en.e_ref ? en.c_energy : nullptr);
    fm_reduce(partial_a, ra, n_params, {{o.A, o.A + S * F},                      // A
                                        {o.U1[0], o.c2[0] + F},                 // U1, c1, U2, c2
                                        {o.R1, o.e0 + S}}, grad, s);            // R1, d1, R2, d2, e0
    const int ge = fm_edge_ctas(n);
    a.atoms_per_cta = fm_edge_atoms(n, 1);               // the gradient pass: one CTA per SM
    if (tensor_cores) {
        if (K == 8) grad_edge_tc_go<32, 8>(a, g, mbar_psi, mdotbar_psi, ubar, partial_e, n_params, status, s);
        else grad_edge_tc_go<32, 16>(a, g, mbar_psi, mdotbar_psi, ubar, partial_e, n_params, status, s);
    } else {
        if (K == 8) grad_edge_go<32, 8>(a, g, mbar_psi, mdotbar_psi, ubar, partial_e, n_params, s);
        else grad_edge_go<32, 16>(a, g, mbar_psi, mdotbar_psi, ubar, partial_e, n_params, s);
    }
    fm_reduce(partial_e, ge, n_params, {{o.W1[0], o.b2[0] + F}}, grad, s);       // W1, b1, W2, b2
    const int gi = fm_input_ctas(n);
    k_fm_input<<<gi, kAtomWarps * 32, 0, s>>>(a, ubar, partial_a, n_params);
    fm_reduce(partial_a, gi, n_params, {{o.A, o.A + S * F},                      // A
                                        {o.W_in[0], o.W_in[0] + F * F}}, grad, s);   // W_in
    count_launch(9);
}

}  // namespace dmts
