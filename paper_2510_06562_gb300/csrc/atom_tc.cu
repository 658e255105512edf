// Per-atom MLPs of the potential on the 5th-generation tensor cores (the
// BF16 precision mode): the same stages as the FP32 kernels of atom_mlp.cu,
//
//   forward, layer l:   z = m U1 + c1;  h <- h + SiLU(z) U2 + c2;
//                       l < L-1:  u^{l+1} = h W_in^{l+1}
//                       l = L-1:  q = h R1 + d1;  E_i = SiLU(q) . R2 + d2 + e0[Z_i] + E_rep,i;
//                                 gh = (SiLU'(q) * R2) R1^T;  mbar^l = ((gh U2^T) * SiLU'(z)) U1^T
//   backward, layer l >= 1:  gh <- gh + ubar^l W_in^{l T};
//                            mbar^{l-1} = ((gh U2^{l-1 T}) * SiLU'(z^{l-1})) U1^{l-1 T}
//
// with every [128 atoms x F] x [F x F] product one group of tcgen05.mma.
// A CTA takes 128 atoms (tensor-memory lanes) with F / 16 threads each:
// thread x handles atom x mod 128 and the 16 features 16 (x / 128) .. +15
// (warp w reads lanes 32 (w mod 4) .. +31 of the accumulator), so the
// epilogues are elementwise; only the energy sums a row's F / 16 partial
// sums, through shared memory.
//
// Global rows move through shared-memory staging buffers with coalesced
// 16-byte accesses (consecutive threads, consecutive pieces of the CTA's
// contiguous rows): the inputs by asynchronous copies at the start, each
// output right after the barrier that follows its epilogue, while the next
// MMAs run. Staged rows are padded to F + 4 floats, so the 16-byte accesses
// of a warp's 32 rows at the same feature fall into distinct banks; in the
// epilogues a thread reads and writes only its own 16-float chunk of a row.
//
// Precision: every operand is split into two BF16 parts, x = hi + lo with
// hi = bf16(x) and lo = bf16(x - hi), and a product is accumulated in FP32
// as A_hi B_hi + A_lo B_hi + A_hi B_lo (the dropped A_lo B_lo term and the
// rounding of lo leave a relative error near 2^-16 per product, against
// 2^-8 for plain BF16 operands).
//
// Weights: per layer the six matrices W_in, U1, U2 (as B operands of X W)
// and their transposes (B operands of X W^T), then R1 and R1^T, each as a
// hi tile and a lo tile in the K-major layout of umma.cuh, prepared on the
// host at every parameter upload. A stage's tiles stream into one of two
// shared-memory buffers by a bulk asynchronous copy (completion on an
// mbarrier), issued two stages ahead.
#include <algorithm>

#include "internal.cuh"
#include "umma.cuh"

namespace dmts {

namespace {

using namespace umma;

constexpr int kA = 128;                      // atoms per CTA = TMEM lanes
constexpr uint32_t kWait = 1u << 22;         // bounded mbarrier polls

template <int F>
struct AtcSmem {
    unsigned char ahi[kA * F * 2];           // A operand, high BF16 part
    unsigned char alo[kA * F * 2];           //             low part
    unsigned char b[2][2 * F * F * 2];       // two stage buffers: B hi tile, then B lo tile
    float bias[4][F];                        // c1, c2 of this layer; d1, R2 (last layer)
    float ered[F / 16][kA];                  // partial energy sums (last layer)
    float io[3][kA * (F + 4)];               // staged global rows (inputs, then outputs in place)
    uint64_t mbar_b[2];                      // bulk-copy completion, per buffer
    uint64_t mbar_mma;                       // MMA completion
    uint32_t taddr;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// Bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16);
// completes transaction bytes on mbar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}

template <int F>
constexpr int kIoStride = F + 4;                     // floats per staged row

// This thread's 16-float chunk c of staged row t.
template <int F>
__device__ __forceinline__ void io_ld(const float* buf, int t, int c, float* v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(buf + t * kIoStride<F> + c + 4 * q);
        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
}
template <int F>
__device__ __forceinline__ void io_st(float* buf, int t, int c, const float* v) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(buf + t * kIoStride<F> + c + 4 * q) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}

// All threads: the CTA's rows 0 .. nrows - 1 of a global [.][F] array (row
// stride F) into a staging buffer (row stride F + 4), asynchronously, or a
// staging buffer out to global.
template <int F, int NT>
__device__ __forceinline__ void rows_in(float* buf, const float* src, int nrows) {
    for (int k = threadIdx.x; k < nrows * (F / 4); k += NT)
        cp_async16(buf + (k / (F / 4)) * kIoStride<F> + (k % (F / 4)) * 4, src + (size_t)k * 4);
}
template <int F, int NT>
__device__ __forceinline__ void rows_out(float* dst, const float* buf, int nrows) {
    for (int k = threadIdx.x; k < nrows * (F / 4); k += NT)
        reinterpret_cast<float4*>(dst)[k] =
            *reinterpret_cast<const float4*>(buf + (k / (F / 4)) * kIoStride<F> + (k % (F / 4)) * 4);
}

__device__ __forceinline__ float sig(float x) { return 1.0f / (1.0f + __expf(-x)); }

// x = hi + lo, both BF16 (hi round-to-nearest, lo the rounded remainder)
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Row t, features c .. c + 15, into the A operand (hi and lo tiles).
template <int F>
__device__ __forceinline__ void put_a(AtcSmem<F>& S, int t, int c, const float* v) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(v[8 * h + 2 * q], h0, l0);
            split_bf16(v[8 * h + 2 * q + 1], h1, l1);
            __nv_bfloat162 ph(h0, h1), pl(l0, l1);
            wh[q] = *reinterpret_cast<uint32_t*>(&ph);
            wl[q] = *reinterpret_cast<uint32_t*>(&pl);
        }
        const uint32_t off = tile_offset(t, c + 8 * h, F);
        *reinterpret_cast<uint4*>(S.ahi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4*>(S.alo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
}

template <int F>
__device__ __forceinline__ void zero_a(AtcSmem<F>& S, int t) {
#pragma unroll
    for (int k = 0; k < F; k += 8) {
        *reinterpret_cast<uint4*>(S.ahi + tile_offset(t, k, F)) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(S.alo + tile_offset(t, k, F)) = make_uint4(0, 0, 0, 0);
    }
}

// 16 features as BF16 into the u (half 0) or mbar (half 1) part of an
// interleaved row of the tensor-core edge backward (per 16 features 16 u
// values then 16 mbar values; F * 4 bytes per atom).
__device__ __forceinline__ void st16_um(unsigned char* __restrict__ row, int c, int half, const float* v) {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<uint32_t*>(&p);
    }
    uint4* d = reinterpret_cast<uint4*>(row + c * 4 + half * 32);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Weight slots: per layer l, 6 l + {W_in, U1, U2, W_in^T, U1^T, U2^T}; then
// 6 L + {R1, R1^T}. Slot bytes: hi tile then lo tile, F x F BF16 each.
enum { kWin = 0, kU1 = 1, kU2 = 2, kWinT = 3, kU1T = 4, kU2T = 5 };

__device__ __forceinline__ int slot_of(int s, int bwd, int last, int l, int L) {
    if (bwd) return s == 0 ? 6 * l + kWinT : (s == 1 ? 6 * (l - 1) + kU2T : 6 * (l - 1) + kU1T);
    switch (s) {
        case 0: return 6 * l + kU1;
        case 1: return 6 * l + kU2;
        case 2: return last ? 6 * L : 6 * (l + 1) + kWin;
        case 3: return 6 * L + 1;
        case 4: return 6 * l + kU2T;
        default: return 6 * l + kU1T;
    }
}

// One CTA: atoms blockIdx.x * 128 + threadIdx.x. bwd = 0: forward of layer
// p.layer (3 stages, or 6 for the last layer); bwd = 1: backward tail of
// layer p.layer >= 1 (3 stages). msg: the per-atom sums of the edge pass
// (messages m^l, or ubar^l).
template <int F>
__global__ void __launch_bounds__(kA * (F / 16)) k_atom_tc(PotArgs p, const float* __restrict__ msg, int bwd,
                                                          int* status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    AtcSmem<F>& S = *reinterpret_cast<AtcSmem<F>*>(smraw);
    constexpr uint32_t kTile = 2u * F * F * 2u;
    constexpr int NT = kA * (F / 16);
    const int x = threadIdx.x, warp = x >> 5;
    const int t = x & (kA - 1);                        // atom row (TMEM lane)
    const int g = x / kA;                              // feature chunk
    const int c = 16 * g;
    const int i = blockIdx.x * kA + t;
    const bool live = i < p.n_atoms;
    const int l = p.layer, L = p.n_layers;
    const int last = (!bwd && l == L - 1) ? 1 : 0;
    const int ns = (!bwd && last) ? 6 : 3;
    const int nrows = min(kA, p.n_atoms - (int)blockIdx.x * kA);
    const size_t roff = (size_t)blockIdx.x * kA * F;
    static_assert((kIoStride<F> * 4) % 16 == 0, "staged rows start on 16-byte boundaries");

    // inputs: messages or ubar (io 0), h or gh (io 1), z^{l-1} (io 2, backward)
    rows_in<F, NT>(S.io[0], msg + roff, nrows);
    rows_in<F, NT>(S.io[1], (bwd ? p.gh : p.h_in) + roff, nrows);
    if (bwd) rows_in<F, NT>(S.io[2], p.z_prev + roff, nrows);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int issued = 0, waited = 0;                        // thread 0: weight copies issued / consumed
    if (x == 0) {
        mbar_init(&S.mbar_b[0], 1);
        mbar_init(&S.mbar_b[1], 1);
        mbar_init(&S.mbar_mma, 1);
        for (int s = 0; s < 2 && s < ns; ++s) {        // the first two stages' weights
            mbar_expect_tx(&S.mbar_b[s], kTile);
            bulk_g2s(S.b[s], p.at + (size_t)slot_of(s, bwd, last, l, L) * kTile, kTile, &S.mbar_b[s]);
            ++issued;
        }
    }
    if (warp == 0) tmem_alloc(&S.taddr, 2 * F);
    if (!bwd)
        for (int k = x; k < F; k += NT) {
            S.bias[0][k] = __ldg(p.P + p.off.c1[l] + k);
            S.bias[1][k] = __ldg(p.P + p.off.c2[l] + k);
            if (last) {
                S.bias[2][k] = __ldg(p.P + p.off.d1 + k);
                S.bias[3][k] = __ldg(p.P + p.off.R2 + k);
            }
        }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tD = S.taddr + c, tStash = S.taddr + F + c;   // this thread's columns
    const uint32_t lane = (uint32_t)(32 * (warp & 3)) << 16;
    bool mma_out = false;                              // thread 0: an MMA group not yet seen complete
    double e_const = 0.0;                              // d2 + e0[Z_i] + E_rep,i (last layer)
    if (last && live && g == 0)
        e_const = (double)__ldg(p.P + p.off.d2) + (double)__ldg(p.P + p.off.e0 + p.species[i]) + (double)p.erep[i];
    bool ok = true;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();                                   // every thread's input copies have landed
    {
        // stage 0's A operand: this atom's message (forward) or ubar (backward) chunk
        float v[16];
        io_ld<F>(S.io[0], t, c, v);
        put_a<F>(S, t, c, v);
    }

    uint32_t ph = 0;
    float* out_dst = nullptr;                          // output of the previous stage, staged in io[out_buf]
    int out_buf = 0;
    for (int s = 0; s < ns; ++s) {
        if (x == 0 && ok) {
            ok = mbar_wait(&S.mbar_b[s & 1], (uint32_t)((s >> 1) & 1), kWait);
            waited += ok ? 1 : 0;
        }
        fence_proxy_async();
        fence_before_sync();
        ok = __syncthreads_and(ok);
        fence_after_sync();
        if (!ok) break;
        if (x == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, F);
            const uint32_t ah = smem_u32(S.ahi), al = smem_u32(S.alo);
            const uint32_t bh = smem_u32(S.b[s & 1]), bl = bh + F * F * 2;
#pragma unroll
            for (int kk = 0; kk < F / 16; ++kk) {
                const uint64_t dah = make_desc(ah + kk * 256, 128, F * 16), dal = make_desc(al + kk * 256, 128, F * 16);
                const uint64_t dbh = make_desc(bh + kk * 256, 128, F * 16), dbl = make_desc(bl + kk * 256, 128, F * 16);
                mma_bf16(S.taddr, dah, dbh, idesc, kk > 0 ? 1u : 0u);
                mma_bf16(S.taddr, dal, dbh, idesc, 1u);
                mma_bf16(S.taddr, dah, dbl, idesc, 1u);
            }
            mma_commit(&S.mbar_mma);
            mma_out = true;
        }
        if (out_dst) rows_out<F, NT>(out_dst + roff, S.io[out_buf], nrows);   // the previous stage's output
        out_dst = nullptr;
        // the last layer's energy: the previous stage left the partial sums
        if (last && s == 3 && g == 0 && live) {
            float e = 0.f;
#pragma unroll
            for (int k = 0; k < F / 16; ++k) e += S.ered[k][t];
            p.Ei[i] = (double)e + e_const;
        }
        ok = mbar_wait(&S.mbar_mma, ph, kWait);
        ph ^= 1u;                                      // a group not seen complete has parity ph ^ 1
        if (x == 0 && ok) mma_out = false;
        fence_after_sync();
        if (!ok) continue;                             // the next barrier ends the loop
        // this stage's buffer is free: fetch the tiles of stage s + 2 into it
        if (x == 0 && s + 2 < ns) {
            mbar_expect_tx(&S.mbar_b[s & 1], kTile);
            bulk_g2s(S.b[s & 1], p.at + (size_t)slot_of(s + 2, bwd, last, l, L) * kTile, kTile, &S.mbar_b[s & 1]);
            ++issued;
        }
        const int code = bwd ? 10 + s : (s == 2 && !last ? 9 : s);
        float v[16], o[16], pre[16];
        tmem_ld16(tD + lane, v);
        switch (code) {
            case 0: {                                  // z = m U1 + c1; A = SiLU(z)
                float dz[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float z = v[q] + S.bias[0][c + q];
                    const float sg = sig(z);
                    v[q] = z;
                    o[q] = z * sg;
                    dz[q] = fmaf(o[q], 1.f - sg, sg);  // SiLU'(z)
                }
                io_st<F>(S.io[0], t, c, v);
                out_dst = p.z;
                out_buf = 0;
                if (last) {
                    tmem_st16(tStash + lane, dz);
                    tmem_st_wait();
                }
                put_a<F>(S, t, c, o);
                break;
            }
            case 1: {                                  // h <- h + SiLU(z) U2 + c2; A = h
                io_ld<F>(S.io[1], t, c, pre);
#pragma unroll
                for (int q = 0; q < 16; ++q) o[q] = pre[q] + (v[q] + S.bias[1][c + q]);
                io_st<F>(S.io[1], t, c, o);
                out_dst = p.h;
                out_buf = 1;
                put_a<F>(S, t, c, o);
                break;
            }
            case 9:                                    // u^{l+1} = h W_in^{l+1}
                io_st<F>(S.io[2], t, c, v);
                out_dst = p.u_next;
                out_buf = 2;
                if (live && p.um_u_out) st16_um(p.um_u_out + (size_t)i * F * 4, c, 0, v);
                break;
            case 2: {                                  // q = h R1 + d1; energy; A = SiLU'(q) R2
                float e = 0.f;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float xq = v[q] + S.bias[2][c + q], r2 = S.bias[3][c + q];
                    const float sg = sig(xq);
                    e += xq * sg * r2;
                    o[q] = sg * (1.f + xq * (1.f - sg)) * r2;
                }
                S.ered[g][t] = e;
                put_a<F>(S, t, c, o);
                break;
            }
            case 3:                                    // gh = gq R1^T; A = gh
                io_st<F>(S.io[2], t, c, v);
                out_dst = p.gh;
                out_buf = 2;
                put_a<F>(S, t, c, v);
                break;
            case 4: {                                  // A = (gh U2^T) * SiLU'(z)
                float dz[16];
                tmem_ld16(tStash + lane, dz);
#pragma unroll
                for (int q = 0; q < 16; ++q) o[q] = v[q] * dz[q];
                put_a<F>(S, t, c, o);
                break;
            }
            case 5:                                    // mbar^l = gz U1^T
            case 12:                                   // mbar^{l-1} = gz U1^{l-1 T}
                io_st<F>(S.io[0], t, c, v);
                out_dst = p.mbar_out;
                out_buf = 0;
                if (live && p.um_mbar_out) st16_um(p.um_mbar_out + (size_t)i * F * 4, c, 1, v);
                break;
            case 10: {                                 // gh <- gh + ubar W_in^{l T}; A = gh
                io_ld<F>(S.io[1], t, c, pre);
#pragma unroll
                for (int q = 0; q < 16; ++q) o[q] = pre[q] + v[q];
                io_st<F>(S.io[1], t, c, o);
                out_dst = p.gh;
                out_buf = 1;
                put_a<F>(S, t, c, o);
                break;
            }
            case 11: {                                 // A = (gh U2^{l-1 T}) * SiLU'(z^{l-1})
                io_ld<F>(S.io[2], t, c, pre);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float z = pre[q];
                    const float sg = sig(z);
                    o[q] = v[q] * sg * (1.f + z * (1.f - sg));
                }
                put_a<F>(S, t, c, o);
                break;
            }
            default:
                break;
        }
    }
    // the last stage's output; after a failed wait, the CTA's copies and MMAs
    // in flight complete before it leaves
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    if (ok && out_dst) rows_out<F, NT>(out_dst + roff, S.io[out_buf], nrows);
    bool drained = true;                               // status bit 1: something still in flight
    if (x == 0) {
        while (waited < issued) {
            if (!mbar_wait(&S.mbar_b[waited & 1], (uint32_t)((waited >> 1) & 1), kWait)) {
                drained = false;
                break;
            }
            ++waited;
        }
        if (mma_out && !mbar_wait(&S.mbar_mma, ph ^ 1u, kWait)) drained = false;
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(S.taddr, 2 * F);
    if (!ok && x == 0) atomicOr(status, drained ? 1 : 3);
}

template <int F>
void atom_tc_go(const PotArgs& p, const float* msg, int bwd, int* status, cudaStream_t s) {
    const int smem = (int)sizeof(AtcSmem<F>);
    smem_opt_in((const void*)k_atom_tc<F>, smem);
    k_atom_tc<F><<<(p.n_atoms + kA - 1) / kA, kA * (F / 16), smem, s>>>(p, msg, bwd, status);
}

}  // namespace

void launch_atom_fwd_tc(const PotArgs& p, int F, const float* msg, int* status, cudaStream_t s) {
    if (p.n_atoms == 0) return;
    if (F == 64) atom_tc_go<64>(p, msg, 0, status, s);
    else atom_tc_go<32>(p, msg, 0, status, s);
    count_launch();
}

void launch_atom_bwd_tc(const PotArgs& p, int F, const float* ubar, int* status, cudaStream_t s) {
    if (p.n_atoms == 0) return;
    if (F == 64) atom_tc_go<64>(p, ubar, 1, status, s);
    else atom_tc_go<32>(p, ubar, 1, status, s);
    count_launch();
}

size_t atom_tile_bytes(int F, int L) { return (size_t)(6 * L + 2) * 2 * F * F * 2; }

}  // namespace dmts
