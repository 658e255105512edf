// BF16 tensor-core path of the potential (DMTS_BF16_MLP): the per-edge filter
// MLP runs on the 5th-generation tensor cores (tcgen05.mma, BF16 operands in
// shared or tensor memory, FP32 accumulators in tensor memory); edge
// geometry, message sums and forces stay FP32.
//
// The pair list is cut into fixed tiles of 128 pairs, taken round-robin by
// persistent CTAs: one pair per thread and per TMEM lane, so after each MMA a
// thread loads its own pair's feature row from TMEM. A CTA of 4 warps has one
// tile in flight; the F = 64 backward pass has two, in two groups of 4 warps
// sharing the weight tiles. Per-atom sums (messages, or the adjoint ubar,
// forces and virial) of rows that start and end in a tile go to global memory
// directly; rows split across tiles are summed in tile order by a fix-up
// pass. The per-atom MLPs run in their own kernels.
//   forward, per tile:  A1 = basis (128 x 16)           D1 = A1 W1        (hidden pre-activation)
//                       A2 = SiLU(D1 + b1) (128 x F)    D2 = A2 W2        (filter, w = fc (D2 + b2))
//   backward, per tile: D1 = A1 W1, D4 = A1' W1 (basis derivative), D2 = SiLU(D1 + b1) W2,
//                       g = mbar_i u_j + mbar_j u_i,  D3 = g W2^T,
//                       dE/dd = fc' (g . (D2 + b2)) + fc sum_k D3_k SiLU'(D1_k + b1_k) D4_k.
// The MMAs are issued by one thread; completion is signalled through an
// mbarrier (bounded waits: a wait that gives up sets the timeout flag and the
// kernel finishes without further MMAs, freeing its tensor memory).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "f32x2.cuh"
#include "internal.cuh"
#include "umma.cuh"

namespace dmts {

namespace {

using namespace umma;

constexpr int kT = 128;          // threads per CTA = edges per tile = TMEM lanes
constexpr int kKP = 16;          // radial functions padded to one MMA K step
constexpr uint32_t kWaitIter = 1u << 22;

// After a completion wait that gave up: the issuing thread waits, again with
// a bound, for the MMA group it committed last (parity pend) if it has not
// seen that group complete, so that the tensor memory those MMAs write is not
// freed under them. Returns false if this wait gives up too.
__device__ __forceinline__ bool drain_mma(bool mma_out, uint64_t* mbar, uint32_t pend) {
    return !mma_out || mbar_wait(mbar, pend, kWaitIter);
}

constexpr f2::f32x2 kHalf2 = 0x3F0000003F000000ull;        // (0.5f, 0.5f)
constexpr f2::f32x2 kMinusHalf2 = 0xBF000000BF000000ull;   // (-0.5f, -0.5f)

// tanh(x / 2) of both halves (the hardware approximation, one per half)
__device__ __forceinline__ f2::f32x2 tanh_half(f2::f32x2 x) {
    const f2::f32x2 h = f2::mul(x, kHalf2);
    float t0, t1;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(f2::lo(h)));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(f2::hi(h)));
    return f2::pack(t0, t1);
}

__device__ __forceinline__ float sigmoid_fast(float x) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * x));
    return fmaf(0.5f, t, 0.5f);
}

// Asynchronous 16-byte global -> shared copies; the issuing thread waits for
// its own copies with cp_async_wait(). They bypass L1 (a gathered row is
// reused by other tiles much later, if at all), which leaves the few KB of
// L1 beside the shared-memory carve-out to the receiving atoms' rows.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst_smem)), "l"(src) : "memory");
}

// Pull the 128-byte lines of an F-float row into L1 ahead of its use.
template <int F>
__device__ __forceinline__ void prefetch_row_l1(const float* row) {
#pragma unroll
    for (int k = 0; k < F * 4; k += 128) asm volatile("prefetch.global.L1 [%0];" :: "l"(row + k / 4));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Per-edge feature rows in shared memory: [kT][F] floats, unpadded, with the
// 16-byte chunks of row e XOR-swizzled by (e mod 8). One thread reading its
// own row chunk by chunk, and one warp reading 32 consecutive floats of one
// row, both touch 32 distinct banks.
template <int F>
__device__ __forceinline__ int prow(int e, int f) {
    return e * F + ((((f >> 2) ^ (e & 7))) << 2) + (f & 3);
}

// Gather row j of src (F floats per row) for each of the warp's 32 edges into
// the swizzled buffer. Each row is copied by F/4 consecutive lanes, 16 bytes
// each, so one warp instruction reads 32 / (F/4) whole rows: the loads are
// coalesced per row instead of one scattered row per lane.
template <int F>
__device__ __forceinline__ void gather_rows(float* buf, const float* __restrict__ src, int j, int tid) {
    constexpr int TPR = F / 4;
    constexpr int RPI = 32 / TPR;
    const int lane = tid & 31, w0 = tid & ~31;       // tid: the thread's edge within the tile
    const int sub = lane / TPR, ch = lane % TPR;
#pragma unroll
    for (int rr = 0; rr < 32; rr += RPI) {
        const int je = __shfl_sync(0xffffffffu, j, rr + sub);
        const int e = w0 + rr + sub;
        cp_async16(buf + e * F + ((ch ^ (e & 7)) << 2), src + (size_t)je * F + ch * 4);
    }
}

// Edge indices and fixed-point positions of one tile edge, loaded one tile
// ahead; rp is the row of the pair before it (-1 for the first pair).
struct EdgeIn {
    int j, i, rp;
    uint4 qj, qi;
};

__device__ __forceinline__ void load_idx(const PotArgs& a, long long e, long long e_end, EdgeIn& x) {
    if (e < e_end) {
        x.j = DMTS_IDX(__ldg(a.col + e), a.n_atoms, a.check);
        x.i = DMTS_IDX(__ldg(a.recv + e), a.n_atoms, a.check);
        x.rp = e > 0 ? __ldg(a.recv + e - 1) : -1;
    } else {
        x.j = -1;
        x.i = -1;
        x.rp = -1;
    }
}

__device__ __forceinline__ void load_pos(const PotArgs& a, EdgeIn& x) {
    if (x.j >= 0) {
        x.qj = __ldg(a.q + x.j);
        x.qi = __ldg(a.q + x.i);
    }
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

// Bessel basis (K <= 16 functions, padded with zeros to 16) and its derivative,
// from inv_d = 1/d. The angle pi d / rc lies in [0, pi], where the hardware
// sine/cosine approximations are accurate to ~1e-6 absolute, far below the
// BF16 rounding the basis undergoes next.
// KC > 0: the number of functions as a compile-time constant (the terms
// past it, and the recurrence steps that feed only them, compile away);
// KC = 0: K at run time.
template <int KC>
__device__ __forceinline__ void basis16(float d, float inv_d, int K, float pi_over_rc, float pref, float* e,
                                        float* de, float& fc, float& dfc) {
    float s1, c1;
    __sincosf(d * pi_over_rc, &s1, &c1);
    // sin(k t) and cos(k t), t = pi d / rc, by the Chebyshev recurrence
    float sk[kKP], ck[kKP];
    sk[0] = s1;
    ck[0] = c1;
    const float c2 = 2.f * c1;
#pragma unroll
    for (int k = 1; k < kKP; ++k) {
        sk[k] = c2 * sk[k - 1] - (k > 1 ? sk[k - 2] : 0.f);
        ck[k] = c2 * ck[k - 1] - (k > 1 ? ck[k - 2] : 1.f);
    }
    // e_k = A sin(k t), e'_k = A (k pi / rc) cos(k t) - (A / d) sin(k t), A = pref / d;
    // two functions per packed FP32 operation
    const float A = pref * inv_d;
    const f2::f32x2 A2 = f2::splat(A), mB2 = f2::splat(-A * inv_d), W2 = f2::splat(A * pi_over_rc);
#pragma unroll
    for (int k = 0; k < kKP; k += 2) {
        const bool on0 = KC > 0 ? k < KC : k < K, on1 = KC > 0 ? k + 1 < KC : k + 1 < K;
        const f2::f32x2 S = f2::pack(sk[k], sk[k + 1]);
        const f2::f32x2 E = f2::mul(A2, S);
        e[k] = on0 ? f2::lo(E) : 0.f;
        e[k + 1] = on1 ? f2::hi(E) : 0.f;
        if (de) {
            const f2::f32x2 DE = f2::fma(f2::mul(W2, f2::pack((float)(k + 1), (float)(k + 2))),
                                         f2::pack(ck[k], ck[k + 1]), f2::mul(mB2, S));
            de[k] = on0 ? f2::lo(DE) : 0.f;
            de[k + 1] = on1 ? f2::hi(DE) : 0.f;
        }
    }
    fc = 0.5f * (c1 + 1.0f);
    dfc = -0.5f * pi_over_rc * s1;
}

// ------------------------------------------------------------ segmented sums
// Rows (receiving atoms) are contiguous runs of edges. Vector sums (F values
// per edge, in sP[e][f]): every warp sums its 32 edges sequentially, each lane
// F / 32 adjacent features; rows that start and end inside the warp are complete and are
// written to global memory directly, the warp's first and last row segments
// go to two slots. Scalar sums (NV values per edge): a segmented shuffle scan
// per warp, every row segment to a slot. The slots are then merged in edge
// order by one thread per value, carrying the open row across tiles.
template <int F>
struct alignas(16) VecSlots {
    float v[4][2][F];
    int row[4][2];
};

template <int F>
__device__ __forceinline__ void warp_vec_segments(const float* __restrict__ sP, int myrow,
                                                  VecSlots<F>* __restrict__ vs, float* __restrict__ out, int a0,
                                                  int tid) {
    constexpr int VW = F / 32;                     // consecutive features per lane (one 4- or 8-byte access)
    static_assert(VW == 1 || VW == 2, "F must be 32 or 64");
    const int w = tid >> 5, lane = tid & 31;       // tid: the thread's edge within the tile
    const int f0 = VW * lane;
    // row of every edge of the warp (myrow: this lane's); segment starts as a warp-uniform bit mask
    const int prev = __shfl_up_sync(0xffffffffu, myrow, 1);
    const unsigned int valid = __ballot_sync(0xffffffffu, myrow >= 0);
    const unsigned int starts = __ballot_sync(0xffffffffu, myrow >= 0 && (lane == 0 || prev != myrow));
    const int n_valid = __popc(valid);             // valid edges form a prefix
    if (lane == 0) {
        vs->row[w][0] = -1;
        vs->row[w][1] = -1;
    }
    const float* base = sP + (32 * w) * F;
    auto put = [&](float* dst, const float* v) {
        if constexpr (VW == 2) *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
        else *dst = v[0];
    };
    // one pass per segment (warp-uniform bounds), its edges summed in order
    unsigned int rem = starts;
    for (int seg = 0; rem; ++seg) {
        const int e0 = __ffs(rem) - 1;
        rem &= rem - 1u;
        const int e1 = rem ? __ffs(rem) - 1 : n_valid;
        float acc[VW];                             // e0 < e1: the segment has an edge
        if constexpr (VW == 2) {
            f2::f32x2 a2 = *reinterpret_cast<const f2::f32x2*>(base + prow<F>(e0, f0));
#pragma unroll 4
            for (int e = e0 + 1; e < e1; ++e) a2 = f2::add(a2, *reinterpret_cast<const f2::f32x2*>(base + prow<F>(e, f0)));
            acc[0] = f2::lo(a2);
            acc[1] = f2::hi(a2);
        } else {
            acc[0] = base[prow<F>(e0, f0)];
#pragma unroll 4
            for (int e = e0 + 1; e < e1; ++e) acc[0] += base[prow<F>(e, f0)];
        }
        const int r = __shfl_sync(0xffffffffu, myrow, e0);
        if (seg == 0) {                            // may continue a row of the previous warp
            put(&vs->v[w][0][f0], acc);
            if (lane == 0) vs->row[w][0] = r;
        } else if (e1 == n_valid) {                // may continue into the next warp
            put(&vs->v[w][1][f0], acc);
            if (lane == 0) vs->row[w][1] = r;
        } else {
            put(out + (size_t)(a0 + r) * F + f0, acc);
        }
    }
}

// Pair tiles. Tile t holds pairs [tb, te) = [128 t, min(128 t + 128, E)).
// A row's segment in the tile is complete when the row starts and ends
// inside it; otherwise the tile's first segment (a row begun in an earlier
// tile) goes to the tile's "first" carry slot and its last segment (a row
// that continues into later tiles) to its "last" slot. k_tile_fixup then
// gives each split row the sum of its head tile's last slot and the later
// tiles' first slots, in tile order. Carry slots hold F vector values then
// the scalar values of the pass. prev_row / next_row are the rows of pairs
// tb - 1 and te (-1 if none): the first segment continues an earlier tile
// iff its row is prev_row, the last continues into a later one iff its row
// is next_row.
struct TileCtx {
    int prev_row, next_row;
    float* cf;                 // this tile's first carry slot
    float* cl;                 // this tile's last carry slot
};

// 0: complete in the tile; 1: continues a row of earlier tiles; 2: a row
// that starts here and continues into later tiles.
__device__ __forceinline__ int seg_route(const TileCtx& t, int r, bool first, bool last) {
    const bool start_in = !first || r != t.prev_row;
    const bool end_in = !last || r != t.next_row;
    return (start_in && end_in) ? 0 : (start_in ? 2 : 1);
}

// Merge the warp slots of one tile in edge order (thread f of the first F
// threads) and route each segment.
template <int F>
__device__ __forceinline__ void merge_tile_vec(const VecSlots<F>* vs, int f, const TileCtx& t,
                                               float* __restrict__ out) {
    int cur = -1;
    float run = 0.f;
    bool first = true;
    auto put = [&](int r, float v, bool fst, bool lst) {
        const int rt = seg_route(t, r, fst, lst);
        if (rt == 0) out[(size_t)r * F + f] = v;
        else if (rt == 1) t.cf[f] = v;
        else t.cl[f] = v;
    };
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int r = vs->row[w][k];
            if (r < 0) continue;
            const float v = vs->v[w][k][f];
            if (r == cur) {
                run += v;
            } else {
                if (cur >= 0) {
                    put(cur, run, first, false);
                    first = false;
                }
                cur = r;
                run = v;
            }
        }
    if (cur >= 0) put(cur, run, first, true);
}

template <int NV>
struct ScalSlots {
    float v[4][32][NV];
    int row[4][32];
    int n[4];
};

template <int NV>
__device__ __forceinline__ void warp_scal_segments(float* val, int row, ScalSlots<NV>* ss, int tid) {
    const int w = tid >> 5, lane = tid & 31;       // tid: the thread's edge within the tile
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int ro = __shfl_up_sync(0xffffffffu, row, off);
        bool same = lane >= off && ro == row;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            float y = __shfl_up_sync(0xffffffffu, val[c], off);
            if (same) val[c] += y;
        }
    }
    int rn = __shfl_down_sync(0xffffffffu, row, 1);
    bool seg_end = row >= 0 && (lane == 31 || rn != row);
    unsigned int ends = __ballot_sync(0xffffffffu, seg_end);
    if (seg_end) {
        int k = __popc(ends & ((1u << lane) - 1u));
        ss->row[w][k] = row;
#pragma unroll
        for (int c = 0; c < NV; ++c) ss->v[w][k][c] = val[c];
    }
    if (lane == 0) ss->n[w] = __popc(ends);
}

// Scalar counterpart of merge_tile_vec (thread c of NV threads): the
// segment ends of the four warps in edge order. store(r, c, v) writes a
// complete row; carries go to slot index F + c.
template <int NV, int F, class Store>
__device__ __forceinline__ void merge_tile_scal(const ScalSlots<NV>* ss, int c, const TileCtx& t, Store store) {
    int cur = -1;
    float run = 0.f;
    bool first = true;
    auto put = [&](int r, float v, bool fst, bool lst) {
        const int rt = seg_route(t, r, fst, lst);
        if (rt == 0) store(r, c, v);
        else if (rt == 1) t.cf[F + c] = v;
        else t.cl[F + c] = v;
    };
    for (int w = 0; w < 4; ++w)
        for (int k = 0; k < ss->n[w]; ++k) {
            const int r = ss->row[w][k];
            const float v = ss->v[w][k][c];
            if (r == cur) {
                run += v;
            } else {
                if (cur >= 0) {
                    put(cur, run, first, false);
                    first = false;
                }
                cur = r;
                run = v;
            }
        }
    if (cur >= 0) put(cur, run, first, true);
}

// Rows without pairs: the thread of the first pair after such rows writes
// their outputs (zeros), and the thread of the last pair writes those of the
// rows after it, so a tiled pass writes every row that does not cross a tile
// boundary. rp: the row of the previous pair (-1 for the first; loaded with
// the pair's indices); vec: F values per row (or null); zero(r) writes the
// row's scalar outputs.
template <int F, class Zero>
__device__ __forceinline__ void fill_empty_rows(int rp, int row, bool last_pair, int n_atoms, float* __restrict__ vec,
                                                Zero zero) {
    auto fill = [&](int r) {
        if (vec) {
            float4* p = reinterpret_cast<float4*>(vec + (size_t)r * F);
#pragma unroll
            for (int k = 0; k < F / 4; ++k) p[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        zero(r);
    };
    for (int r = rp + 1; r < row; ++r) fill(r);
    if (last_pair)
        for (int r = row + 1; r < n_atoms; ++r) fill(r);
}

// Rows split across tiles, after a tiled pass: one warp per tile boundary t
// (1 <= t < tiles). The warp of the first boundary a row crosses gives it the
// sum of its head tile's last carry slot and the later tiles' first slots,
// in tile order. vec_out (F values per atom) may be null; n_scal scalars go
// to erep (kind 0) or to the force and the per-atom virial (kind 1, added
// when accumulate). With no pairs at all, the warps write every row's zeros.
template <int F>
__global__ void __launch_bounds__(256) k_tile_fixup(int n, const int* __restrict__ row_ptr,
                                                    const int* __restrict__ recv, long long e_cap,
                                                    const float* __restrict__ carry, int cw, float* __restrict__ vec_out,
                                                    int n_scal, int kind, float* __restrict__ erep,
                                                    float* __restrict__ force, float* __restrict__ vir6,
                                                    int accumulate, int* check) {
    constexpr int NF = F / 32;
    const int lane = threadIdx.x & 31;
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long E = min((long long)row_ptr[n], e_cap);
    auto put = [&](long long i, const float* v, float sc) {
        if (vec_out)
#pragma unroll
            for (int c = 0; c < NF; ++c) vec_out[(size_t)i * F + lane + 32 * c] = v[c];
        if (lane < n_scal) {
            if (kind == 0) {
                erep[i] = sc;
            } else {
                float* dst = lane < 3 ? force + (size_t)lane * n + i : vir6 + (size_t)i * 6 + lane - 3;
                *dst = accumulate ? *dst + sc : sc;
            }
        }
    };
    float v[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) v[c] = 0.f;
    if (E == 0) {
        const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
        for (long long i = w; i < n; i += nw) put(i, v, 0.f);
        return;
    }
    const long long t = w + 1, n_tiles = (E + 127) >> 7;
    if (t >= n_tiles) return;
    const int r = DMTS_IDX(recv[t << 7], n, check);
    if (recv[(t << 7) - 1] != r) return;                // no row crosses boundary t
    const long long r0 = min((long long)row_ptr[r], e_cap), r1 = min((long long)row_ptr[r + 1], e_cap);
    const long long t0 = r0 >> 7, t1 = (r1 - 1) >> 7;
    if (t0 != t - 1) return;                            // the warp of an earlier boundary sums it
    const float* cl = carry + (2 * t0 + 1) * (long long)cw;
    float sc = 0.f;
#pragma unroll
    for (int c = 0; c < NF; ++c) v[c] = cl[lane + 32 * c];
    if (lane < n_scal) sc = cl[F + lane];
    for (long long u = t0 + 1; u <= t1; ++u) {
        const float* cf = carry + 2 * u * (long long)cw;
#pragma unroll
        for (int c = 0; c < NF; ++c) v[c] += cf[lane + 32 * c];
        if (lane < n_scal) sc += cf[F + lane];
    }
    put(r, v, sc);
}

// Blocks of the fix-up for a pair capacity of e_cap (one warp per possible
// tile boundary, at least one block).
inline int fixup_blocks(long long e_cap) {
    const long long warps = std::max(1LL, (e_cap + 127) / 128);
    return (int)((warps * 32 + 255) / 256);
}

// ------------------------------------------------------------ forward
template <int F>
struct FwdSmem {
    unsigned char w1t[F * kKP * 2];
    unsigned char w2t[F * F * 2];
    unsigned char a1[kT * kKP * 2];     // (the second MMA's A operand lives in tensor memory)
    float b1[F], b2[F];
    float P[kT * F];                    // u_j rows, then messages (swizzled rows)
    VecSlots<F> vs;
    ScalSlots<1> ss;
    uint64_t mbar;
    uint32_t taddr;
};

template <int F, int KC>
__global__ void __launch_bounds__(kT, F == 32 ? 8 : 1) k_edge_fwd_bf16(PotArgs a, int K, int* status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    FwdSmem<F>& S = *reinterpret_cast<FwdSmem<F>*>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int l = a.layer;
    const bool rep_on = l == 0 && a.energy;                // the repulsion energy of layer 0, when read
    const long long E = min((long long)a.row_ptr[a.n_atoms], a.e_cap);
    const long long n_tiles = (E + kT - 1) / kT;
    if ((long long)blockIdx.x >= n_tiles) return;

    // weights: pre-converted BF16 operand tiles (16-byte copies)
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.wt + (size_t)l * a.wt_layer_bytes);
        uint4* d1 = reinterpret_cast<uint4*>(S.w1t);
        uint4* d2 = reinterpret_cast<uint4*>(S.w2t);
        for (int t = tid; t < F * kKP * 2 / 16; t += kT) d1[t] = src[t];
        src += F * kKP * 2 / 16;
        for (int t = tid; t < F * F * 2 / 16; t += kT) d2[t] = src[t];
    }
    for (int t = tid; t < F; t += kT) {
        S.b1[t] = __ldg(a.P + a.off.b1[l] + t);
        S.b2[t] = __ldg(a.P + a.off.b2[l] + t);
    }
    if (tid == 0) mbar_init(&S.mbar, 1);
    if (warp == 0) tmem_alloc(&S.taddr, 2 * F);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = S.taddr;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t idesc = idesc_bf16_f32(128, F);
    const uint32_t sA1 = smem_u32(S.a1);
    const uint32_t sW1T = smem_u32(S.w1t), sW2T = smem_u32(S.w2t);
    uint32_t phase = 0;
    bool ok = true;
    bool mma_out = false;                                  // thread 0: a commit not yet seen complete
    uint32_t pend = 0;                                     // ... and the parity it completes

    const int cw = a.carry_w;
    EdgeIn nx;
    load_idx(a, (long long)blockIdx.x * kT + tid, E, nx);
    load_pos(a, nx);
    for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        {
            const long long tb = tile * kT, te = min(tb + kT, E);
            int prev_row = -1, next_row = -1;              // read by the merges at the end of the tile
            if (tid <= F) {
                if (tb > 0) prev_row = __ldg(a.recv + tb - 1);
                if (te < E) next_row = __ldg(a.recv + te);
            }
            const EdgeIn ex = nx;
            const bool valid = ex.j >= 0;
            const int j = valid ? ex.j : 0;
            const int row = valid ? ex.i : -1;
            if (valid)
                fill_empty_rows<F>(ex.rp, row, tb + tid == E - 1, a.n_atoms, a.msg_out, [&](int r) {
                    if (rep_on) a.erep[r] = 0.f;
                });
            load_idx(a, (tile + gridDim.x) * kT + tid, E, nx);   // next tile's indices
            // the message needs u_j: start copying the warp's rows into P now
            gather_rows<F>(S.P, a.u, j, tid);
            cp_async_commit();
            float fc = 0.f, rep = 0.f;
            {
                float eb[kKP], dfc;
                if (valid) {
                    float3 r = edge_vec(ex.qi, ex.qj, a.frame[ex.qi.w].qscale);
                    float r2 = r.x * r.x + r.y * r.y + r.z * r.z;
                    float inv_d = rsqrtf(r2);
                    float d = r2 * inv_d;
                    basis16<KC>(d, inv_d, K, a.pi_over_rc, a.bessel_pref, eb, nullptr, fc, dfc);
                    if (rep_on) rep = 0.5f * rep_phi(d, a.rep_a, a.rep_inv_rho, a.rep_rc, a.rep_pi_over_rc, nullptr);
                } else {
#pragma unroll
                    for (int k = 0; k < kKP; ++k) eb[k] = 0.f;
                }
                st_row8(S.a1, tid, 0, kKP, eb);
                st_row8(S.a1, tid, 8, kKP, eb + 8);
            }
            fence_proxy_async();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            if (tid == 0) {
                mma_bf16(tmem, make_desc(sA1, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
                mma_commit(&S.mbar);
                mma_out = true;
                pend = phase;
            }
            load_pos(a, nx);                               // next tile's positions
            ok = mbar_wait(&S.mbar, phase, kWaitIter);
            if (tid == 0 && ok) mma_out = false;
            phase ^= 1;
            fence_after_sync();
            // SiLU(a) as BF16 pairs written back over the first F/2 columns of
            // D1 (each block of 16 columns is read before its 8 packed columns
            // are written): the second MMA reads its A operand from there
#pragma unroll
            for (int c = 0; c < F; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + c, v);
                uint32_t pk[8];
#pragma unroll
                for (int q = 0; q < 16; q += 2) {          // two features per packed FP32 operation
                    const f2::f32x2 x = f2::add(f2::pack(v[q], v[q + 1]), *reinterpret_cast<const f2::f32x2*>(S.b1 + c + q));
                    const f2::f32x2 y = f2::mul(x, f2::fma(kHalf2, tanh_half(x), kHalf2));   // SiLU
                    pk[q / 2] = pack_bf16(f2::lo(y), f2::hi(y));
                }
                tmem_st8(tmem + lane_base + c / 2, pk);
            }
            tmem_st_wait();
            fence_before_sync();
            ok = __syncthreads_and(ok);
            fence_after_sync();
            if (tid == 0 && ok) {
#pragma unroll
                for (int kk = 0; kk < F / 16; ++kk)
                    mma_bf16_ta(tmem + F, tmem + kk * 8, make_desc(sW2T + kk * 256, 128, F * 16), idesc, kk > 0);
                mma_commit(&S.mbar);
                mma_out = true;
                pend = phase;
            }
            ok = ok && mbar_wait(&S.mbar, phase, kWaitIter);
            if (tid == 0 && ok) mma_out = false;
            phase ^= 1;
            fence_after_sync();
            cp_async_wait();                               // the warp's u_j rows are in P
            __syncwarp();
            {
                const f2::f32x2 fc2 = f2::splat(fc);
#pragma unroll
                for (int c = 0; c < F; c += 16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + F + c, v);
#pragma unroll
                    for (int q = 0; q < 16; q += 4) {      // message fc (D2 + b2) u_j, two features per operation
                        float* p4 = S.P + prow<F>(tid, c + q);
                        const float4 u4 = *reinterpret_cast<const float4*>(p4);
                        const f2::f32x2* b2 = reinterpret_cast<const f2::f32x2*>(S.b2 + c + q);
                        const f2::f32x2 o01 = f2::mul(f2::mul(fc2, f2::add(f2::pack(v[q], v[q + 1]), b2[0])),
                                                      f2::pack(u4.x, u4.y));
                        const f2::f32x2 o23 = f2::mul(f2::mul(fc2, f2::add(f2::pack(v[q + 2], v[q + 3]), b2[1])),
                                                      f2::pack(u4.z, u4.w));
                        *reinterpret_cast<float4*>(p4) = make_float4(f2::lo(o01), f2::hi(o01), f2::lo(o23), f2::hi(o23));
                    }
                }
            }
            if (rep_on) warp_scal_segments<1>(&rep, row, &S.ss, tid);
            fence_before_sync();
            ok = __syncthreads_and(ok);
            warp_vec_segments<F>(S.P, row, &S.vs, a.msg_out, 0, tid);
            __syncthreads();
            const TileCtx tc{prev_row, next_row, a.carry + 2 * tile * cw, a.carry + (2 * tile + 1) * cw};
            if (tid < F) {
                merge_tile_vec<F>(&S.vs, tid, tc, a.msg_out);
            } else if (tid == F && rep_on) {
                float* erep = a.erep;
                merge_tile_scal<1, F>(&S.ss, 0, tc, [erep](int r, int, float v) { erep[r] = v; });
            }
            // the slots are rewritten only after two more barriers (next tile)
        }
    }
    // after a wait that gave up, the MMAs in flight complete before their
    // tensor memory is freed (status bit 2 if they do not, in time)
    const bool drained = drain_mma(mma_out, &S.mbar, pend);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * F);
    if (!ok && tid == 0) atomicOr(status, drained ? 1 : 3);
}

// ------------------------------------------------------------ backward
// The force (and per-atom virial) of a row without pairs: zero in the pass
// that writes them (the others add).
template <int NV>
__device__ __forceinline__ void zero_force_row(const PotArgs& a, int r) {
    if (a.accumulate) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.force[(size_t)c * a.n_atoms + r] = 0.f;
    if constexpr (NV == 9)
#pragma unroll
        for (int c = 0; c < 6; ++c) a.vir6[(size_t)r * 6 + c] = 0.f;
}

template <int F, int NV>
struct BwdSmem {
    unsigned char w1t[F * kKP * 2];     // B[n][k] = W1[k][n]
    unsigned char w2t[F * F * 2];       // B[n][k] = W2[k][n]
    unsigned char w2n[F * F * 2];       // B[n][k] = W2[n][k]
    unsigned char a14[2 * kT * kKP * 2];  // basis | basis derivative; then the tile's vector and scalar slots
    unsigned char a2[kT * F * 2];       // SiLU hidden, then g
    float b1[F], b2[F];
    // per pair F * 4 bytes: the gathered BF16 row of atom j (per 16 features
    // 16 u_j then 16 mbar_j), overwritten in place by the FP32 ubar message
    // (swizzled 16-byte chunks)
    float G[kT * F];
    uint64_t mbar;
    uint32_t taddr;
};

template <int F>
__host__ __device__ constexpr int scal_slot_offset() { return (int)((sizeof(VecSlots<F>) + 15) / 16 * 16); }

// Eight BF16 values of a 16-byte chunk as FP32 (exact).
__device__ __forceinline__ void unpack_bf16x8(uint4 w, float* v) {
    const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(x[k] << 16);
        v[2 * k + 1] = __uint_as_float(x[k] & 0xffff0000u);
    }
}

// NV = 9: forces and the per-atom virial; NV = 3: forces only.
// L0: the layer-0 pass (a.layer == 0), whose u does not depend on the positions.
template <int F, int NV, int KC, bool L0>
__global__ void __launch_bounds__(kT) k_edge_bwd_bf16(PotArgs a, int K, int* status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    BwdSmem<F, NV>& S = *reinterpret_cast<BwdSmem<F, NV>*>(smraw);
    static_assert(scal_slot_offset<F>() + sizeof(ScalSlots<NV>) <= sizeof(S.a14), "slots must fit the basis tiles");
    // the slots are written once the tile's first MMA (the only reader of the basis tiles) has completed
    VecSlots<F>* vs = reinterpret_cast<VecSlots<F>*>(S.a14);
    ScalSlots<NV>* ss = reinterpret_cast<ScalSlots<NV>*>(S.a14 + scal_slot_offset<F>());
    unsigned char* const a1 = S.a14;
    unsigned char* const a4 = S.a14 + kT * kKP * 2;
    // tensor memory: D1 (then p) | D4, then D2, then D3 (each read before the next MMA overwrites it)
    constexpr int TCOLS = 2 * F;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int l = a.layer;
    const long long E = min((long long)a.row_ptr[a.n_atoms], a.e_cap);
    const long long n_tiles = (E + kT - 1) / kT;
    if ((long long)blockIdx.x >= n_tiles) return;
    constexpr bool need_ubar = !L0;

    {
        const uint4* src = reinterpret_cast<const uint4*>(a.wt + (size_t)l * a.wt_layer_bytes);
        uint4* d1 = reinterpret_cast<uint4*>(S.w1t);
        uint4* d2 = reinterpret_cast<uint4*>(S.w2t);
        uint4* d3 = reinterpret_cast<uint4*>(S.w2n);
        for (int t = tid; t < F * kKP * 2 / 16; t += kT) d1[t] = src[t];
        src += F * kKP * 2 / 16;
        for (int t = tid; t < F * F * 2 / 16; t += kT) d2[t] = src[t];
        src += F * F * 2 / 16;
        for (int t = tid; t < F * F * 2 / 16; t += kT) d3[t] = src[t];
    }
    for (int t = tid; t < F; t += kT) {
        S.b1[t] = __ldg(a.P + a.off.b1[l] + t);
        S.b2[t] = __ldg(a.P + a.off.b2[l] + t);
    }
    if (tid == 0) mbar_init(&S.mbar, 1);
    if (warp == 0) tmem_alloc(&S.taddr, TCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = S.taddr;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t tD1 = tmem, tD4 = tmem + F, tD2 = tmem + F, tD3 = tmem + F;
    const uint32_t idesc = idesc_bf16_f32(128, F);
    const uint32_t sA1 = smem_u32(a1), sA4 = smem_u32(a4), sA2 = smem_u32(S.a2);
    const uint32_t sW1T = smem_u32(S.w1t), sW2T = smem_u32(S.w2t), sW2N = smem_u32(S.w2n);
    uint32_t phase = 0;
    bool ok = true;
    bool mma_out = false;                                  // thread 0: a commit not yet seen complete
    uint32_t pend = 0;                                     // ... and the parity it completes

    const int cw = a.carry_w;
    EdgeIn nx;
    load_idx(a, (long long)blockIdx.x * kT + tid, E, nx);
    load_pos(a, nx);
    for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        {
            const long long tb = tile * kT, te = min(tb + kT, E);
            int prev_row = -1, next_row = -1;              // read by the merges at the end of the tile
            if (tid < F + NV) {
                if (tb > 0) prev_row = __ldg(a.recv + tb - 1);
                if (te < E) next_row = __ldg(a.recv + te);
            }
            const EdgeIn ex = nx;
            const bool valid = ex.j >= 0;
            const int j = valid ? ex.j : 0;
            const int row = valid ? ex.i : -1;
            if (valid)
                fill_empty_rows<F>(ex.rp, row, tb + tid == E - 1, a.n_atoms, need_ubar ? a.msg_out : nullptr,
                                   [&](int r) { zero_force_row<NV>(a, r); });
            load_idx(a, (tile + gridDim.x) * kT + tid, E, nx);   // next tile's indices
            // g needs u_j and mbar_j, the ubar message mbar_j: start the warp's row copies now
            gather_rows<F>(S.G, reinterpret_cast<const float*>(a.um), j, tid);
            cp_async_commit();
            if (valid) {                                   // the receiving atom's rows, read in the second epilogue
                prefetch_row_l1<F>(a.u + (size_t)row * F);
                prefetch_row_l1<F>(a.mbar + (size_t)row * F);
            }
            float fc = 0.f, dfc = 0.f, d = 1.f, rx = 0.f, ry = 0.f, rz = 0.f;
            {
                float eb[kKP], db[kKP];
                if (valid) {
                    const uint4 qi = ex.qi, qj = ex.qj;
                    float3 r = edge_vec(qi, qj, a.frame[qi.w].qscale);
                    float r2 = r.x * r.x + r.y * r.y + r.z * r.z;
                    float inv = rsqrtf(r2);
                    d = r2 * inv;
                    rx = r.x * inv; ry = r.y * inv; rz = r.z * inv;
                    basis16<KC>(d, inv, K, a.pi_over_rc, a.bessel_pref, eb, db, fc, dfc);
                } else {
#pragma unroll
                    for (int k = 0; k < kKP; ++k) { eb[k] = 0.f; db[k] = 0.f; }
                }
                st_row8(a1, tid, 0, kKP, eb);
                st_row8(a1, tid, 8, kKP, eb + 8);
                st_row8(a4, tid, 0, kKP, db);
                st_row8(a4, tid, 8, kKP, db + 8);
            }
            fence_proxy_async();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            if (tid == 0) {
                mma_bf16(tD1, make_desc(sA1, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
                mma_bf16(tD4, make_desc(sA4, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
                mma_commit(&S.mbar);
                mma_out = true;
                pend = phase;
            }
            load_pos(a, nx);                               // next tile's positions
            float se;
            if constexpr (!need_ubar) {
                // Layer 0: u does not depend on the positions, so the pass needs
                // only g . dw/dd. With y = g W2^T, g . phi = SiLU(a) . y + g . b2,
                // and dfc (g . phi) + fc (g . dphi/dd) = sum_k y_k q_k + dfc (g . b2)
                // with q = dfc SiLU(a) + fc SiLU'(a)(e'W1): two dependent MMA
                // groups (D1 | D4, then D3) instead of three. g goes to the MMA
                // operand tile while the first MMAs run.
                cp_async_wait();                           // the warp's u_j | mbar_j rows are in G
                __syncwarp();
                f2::f32x2 gb22 = 0ull;
                {
                    const int i = valid ? row : 0;
                    const float* ui = a.u + (size_t)i * F;
                    const float* mi = a.mbar + (size_t)i * F;
#pragma unroll
                    for (int c = 0; c < F; c += 16) {
                        float4 ui16[4], mi16[4];
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            ui16[qq] = __ldg(reinterpret_cast<const float4*>(ui + c + 4 * qq));
                            mi16[qq] = __ldg(reinterpret_cast<const float4*>(mi + c + 4 * qq));
                        }
                        float g[16], uj[16], mj[16];
                        {
                            uint4 w[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                w[k] = *reinterpret_cast<const uint4*>(S.G + prow<F>(tid, c + 4 * k));
                            unpack_bf16x8(w[0], uj);
                            unpack_bf16x8(w[1], uj + 8);
                            unpack_bf16x8(w[2], mj);
                            unpack_bf16x8(w[3], mj + 8);
                        }
#pragma unroll
                        for (int q = 0; q < 16; q += 4) {
                            const float4 ui4 = ui16[q / 4];
                            const float4 mi4 = mi16[q / 4];
                            const f2::f32x2* b2 = reinterpret_cast<const f2::f32x2*>(S.b2 + c + q);
                            const f2::f32x2 mj01 = f2::pack(mj[q], mj[q + 1]), mj23 = f2::pack(mj[q + 2], mj[q + 3]);
                            const f2::f32x2 g01 = f2::fma(f2::pack(mi4.x, mi4.y), f2::pack(uj[q], uj[q + 1]),
                                                          f2::mul(mj01, f2::pack(ui4.x, ui4.y)));
                            const f2::f32x2 g23 = f2::fma(f2::pack(mi4.z, mi4.w), f2::pack(uj[q + 2], uj[q + 3]),
                                                          f2::mul(mj23, f2::pack(ui4.z, ui4.w)));
                            gb22 = f2::fma(g01, b2[0], gb22);
                            gb22 = f2::fma(g23, b2[1], gb22);
                            g[q] = f2::lo(g01); g[q + 1] = f2::hi(g01);
                            g[q + 2] = f2::lo(g23); g[q + 3] = f2::hi(g23);
                        }
                        st_row8(S.a2, tid, c, F, g);
                        st_row8(S.a2, tid, c + 8, F, g + 8);
                    }
                }
                ok = mbar_wait(&S.mbar, phase, kWaitIter);
                if (tid == 0 && ok) mma_out = false;
                phase ^= 1;
                fence_after_sync();
                const f2::f32x2 fc2 = f2::splat(fc), dfc2 = f2::splat(dfc);
#pragma unroll
                for (int c = 0; c < F; c += 16) {
                    float v[16], tv[16];
                    tmem_ld16x2(tD1 + lane_base + c, v, tD4 + lane_base + c, tv);
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {
                        const f2::f32x2 x = f2::add(f2::pack(v[q], v[q + 1]), *reinterpret_cast<const f2::f32x2*>(S.b1 + c + q));
                        const f2::f32x2 t = tanh_half(x);
                        const f2::f32x2 sg = f2::fma(kHalf2, t, kHalf2), sgc = f2::fma(kMinusHalf2, t, kHalf2);
                        const f2::f32x2 y = f2::mul(x, sg);
                        const f2::f32x2 pd = f2::mul(f2::pack(tv[q], tv[q + 1]), f2::fma(y, sgc, sg));
                        const f2::f32x2 qv = f2::fma(dfc2, y, f2::mul(fc2, pd));
                        // q rounded to BF16, as the two-tile kernel keeps it
                        tv[q] = __bfloat162float(__float2bfloat16_rn(f2::lo(qv)));
                        tv[q + 1] = __bfloat162float(__float2bfloat16_rn(f2::hi(qv)));
                    }
                    tmem_st16(tD1 + lane_base + c, tv);
                }
                tmem_st_wait();
                fence_proxy_async();
                fence_before_sync();
                ok = __syncthreads_and(ok);
                fence_after_sync();
                if (tid == 0 && ok) {
#pragma unroll
                    for (int kk = 0; kk < F / 16; ++kk)
                        mma_bf16(tD3, make_desc(sA2 + kk * 256, 128, F * 16), make_desc(sW2N + kk * 256, 128, F * 16),
                                 idesc, kk > 0);
                    mma_commit(&S.mbar);
                    mma_out = true;
                    pend = phase;
                }
                ok = ok && mbar_wait(&S.mbar, phase, kWaitIter);
                if (tid == 0 && ok) mma_out = false;
                phase ^= 1;
                fence_after_sync();
                f2::f32x2 s22 = 0ull;
#pragma unroll
                for (int c = 0; c < F; c += 16) {
                    float ab[16], pv[16];
                    tmem_ld16x2(tD3 + lane_base + c, ab, tD1 + lane_base + c, pv);
#pragma unroll
                    for (int q = 0; q < 16; q += 2) s22 = f2::fma(f2::pack(ab[q], ab[q + 1]), f2::pack(pv[q], pv[q + 1]), s22);
                }
                se = __fmaf_rn(dfc, f2::lo(gb22) + f2::hi(gb22), f2::lo(s22) + f2::hi(s22));
            } else {
                ok = mbar_wait(&S.mbar, phase, kWaitIter);
                if (tid == 0 && ok) mma_out = false;
                phase ^= 1;
                fence_after_sync();
                // SiLU(a) -> BF16 operand of the next MMA; p = SiLU'(a) (e' W1), the
                // factor the basis-derivative term needs, replaces D1 in tensor memory
#pragma unroll
                for (int c = 0; c < F; c += 16) {
                    float v[16], tv[16];
                    tmem_ld16x2(tD1 + lane_base + c, v, tD4 + lane_base + c, tv);
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {          // two features per packed FP32 operation
                        const f2::f32x2 x = f2::add(f2::pack(v[q], v[q + 1]), *reinterpret_cast<const f2::f32x2*>(S.b1 + c + q));
                        const f2::f32x2 t = tanh_half(x);        // sigmoid(x) = (1 + tanh(x / 2)) / 2
                        const f2::f32x2 sg = f2::fma(kHalf2, t, kHalf2), sgc = f2::fma(kMinusHalf2, t, kHalf2);
                        const f2::f32x2 y = f2::mul(x, sg);
                        const f2::f32x2 pd = f2::mul(f2::pack(tv[q], tv[q + 1]), f2::fma(y, sgc, sg));   // SiLU'(x) T
                        v[q] = f2::lo(y);
                        v[q + 1] = f2::hi(y);
                        // rounded to BF16 as the two-tile kernel keeps it, so the
                        // tuner's choice between the kernels changes no result
                        tv[q] = __bfloat162float(__float2bfloat16_rn(f2::lo(pd)));
                        tv[q + 1] = __bfloat162float(__float2bfloat16_rn(f2::hi(pd)));
                    }
                    st_row8(S.a2, tid, c, F, v);
                    st_row8(S.a2, tid, c + 8, F, v + 8);
                    tmem_st16(tD1 + lane_base + c, tv);
                }
                tmem_st_wait();
                fence_proxy_async();
                fence_before_sync();
                ok = __syncthreads_and(ok);
                fence_after_sync();
                if (tid == 0 && ok) {
#pragma unroll
                    for (int kk = 0; kk < F / 16; ++kk)
                        mma_bf16(tD2, make_desc(sA2 + kk * 256, 128, F * 16), make_desc(sW2T + kk * 256, 128, F * 16),
                                 idesc, kk > 0);
                    mma_commit(&S.mbar);
                    mma_out = true;
                    pend = phase;
                }
                ok = ok && mbar_wait(&S.mbar, phase, kWaitIter);
                if (tid == 0 && ok) mma_out = false;
                phase ^= 1;
                fence_after_sync();
                cp_async_wait();                               // the warp's u_j | mbar_j rows are in G
                __syncwarp();
                f2::f32x2 gphi2 = 0ull;
                {
                    const int i = valid ? row : 0;
                    const f2::f32x2 fc2 = f2::splat(fc);
                    const float* ui = a.u + (size_t)i * F;
                    const float* mi = a.mbar + (size_t)i * F;
#pragma unroll
                    for (int c = 0; c < F; c += 16) {
                        // the receiving atom's rows (shared by most of the warp) before the TMEM load
                        float4 ui16[4], mi16[4];
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            ui16[qq] = __ldg(reinterpret_cast<const float4*>(ui + c + 4 * qq));
                            mi16[qq] = __ldg(reinterpret_cast<const float4*>(mi + c + 4 * qq));
                        }
                        float v[16], g[16], uj[16], mj[16];
                        tmem_ld16(tD2 + lane_base + c, v);
                        {
                            // the four 16-byte chunks of these 16 features: u_j (2), mbar_j (2)
                            uint4 w[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                w[k] = *reinterpret_cast<const uint4*>(S.G + prow<F>(tid, c + 4 * k));
                            unpack_bf16x8(w[0], uj);
                            unpack_bf16x8(w[1], uj + 8);
                            unpack_bf16x8(w[2], mj);
                            unpack_bf16x8(w[3], mj + 8);
                        }
#pragma unroll
                        for (int q = 0; q < 16; q += 4) {      // two features per packed FP32 operation
                            const float4 ui4 = ui16[q / 4];
                            const float4 mi4 = mi16[q / 4];
                            const f2::f32x2* b2 = reinterpret_cast<const f2::f32x2*>(S.b2 + c + q);
                            const f2::f32x2 ph01 = f2::add(f2::pack(v[q], v[q + 1]), b2[0]);
                            const f2::f32x2 ph23 = f2::add(f2::pack(v[q + 2], v[q + 3]), b2[1]);
                            const f2::f32x2 mj01 = f2::pack(mj[q], mj[q + 1]), mj23 = f2::pack(mj[q + 2], mj[q + 3]);
                            // g = mbar_i u_j + mbar_j u_i
                            const f2::f32x2 g01 = f2::fma(f2::pack(mi4.x, mi4.y), f2::pack(uj[q], uj[q + 1]),
                                                          f2::mul(mj01, f2::pack(ui4.x, ui4.y)));
                            const f2::f32x2 g23 = f2::fma(f2::pack(mi4.z, mi4.w), f2::pack(uj[q + 2], uj[q + 3]),
                                                          f2::mul(mj23, f2::pack(ui4.z, ui4.w)));
                            g[q] = f2::lo(g01); g[q + 1] = f2::hi(g01);
                            g[q + 2] = f2::lo(g23); g[q + 3] = f2::hi(g23);
                            gphi2 = f2::fma(g01, ph01, gphi2);
                            gphi2 = f2::fma(g23, ph23, gphi2);
                            // the message replaces the chunks just read (this thread's row only)
                            const f2::f32x2 o01 = f2::mul(f2::mul(fc2, ph01), mj01), o23 = f2::mul(f2::mul(fc2, ph23), mj23);
                            *reinterpret_cast<float4*>(S.G + prow<F>(tid, c + q)) =
                                make_float4(f2::lo(o01), f2::hi(o01), f2::lo(o23), f2::hi(o23));
                        }
                        st_row8(S.a2, tid, c, F, g);
                        st_row8(S.a2, tid, c + 8, F, g + 8);
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
                    mma_commit(&S.mbar);
                    mma_out = true;
                    pend = phase;
                }
                ok = ok && mbar_wait(&S.mbar, phase, kWaitIter);
                if (tid == 0 && ok) mma_out = false;
                phase ^= 1;
                fence_after_sync();
                f2::f32x2 s22 = 0ull;
#pragma unroll
                for (int c = 0; c < F; c += 16) {
                    float ab[16], pv[16];
                    tmem_ld16x2(tD3 + lane_base + c, ab, tD1 + lane_base + c, pv);
#pragma unroll
                    for (int q = 0; q < 16; q += 2) s22 = f2::fma(f2::pack(ab[q], ab[q + 1]), f2::pack(pv[q], pv[q + 1]), s22);
                }
                const float gphi = f2::lo(gphi2) + f2::hi(gphi2), s2 = f2::lo(s22) + f2::hi(s22);
                se = dfc * gphi + fc * s2;
            }
            if (L0 && valid) {
                float dphi;
                (void)rep_phi(d, a.rep_a, a.rep_inv_rho, a.rep_rc, a.rep_pi_over_rc, &dphi);
                se += dphi;
            }
            {
                float val[NV];
                val[0] = se * rx; val[1] = se * ry; val[2] = se * rz;
                if constexpr (NV == 9) {
                    float hv = -0.5f * se * d;
                    val[3] = hv * rx * rx; val[4] = hv * ry * ry; val[5] = hv * rz * rz;
                    val[6] = hv * rx * ry; val[7] = hv * rx * rz; val[8] = hv * ry * rz;
                }
                warp_scal_segments<NV>(val, row, ss, tid);
            }
            fence_before_sync();
            ok = __syncthreads_and(ok);
            if (need_ubar) warp_vec_segments<F>(S.G, row, vs, a.msg_out, 0, tid);
            __syncthreads();
            const TileCtx tc{prev_row, next_row, a.carry + 2 * tile * cw, a.carry + (2 * tile + 1) * cw};
            if (need_ubar && tid < F) {
                merge_tile_vec<F>(vs, tid, tc, a.msg_out);
            } else if (tid >= F && tid < F + NV) {
                float* force = a.force;
                float* vir6 = a.vir6;
                const int n = a.n_atoms, acc = a.accumulate;
                merge_tile_scal<NV, F>(ss, tid - F, tc, [=](int r, int c, float v) {
                    float* dst = c < 3 ? force + (size_t)c * n + r : vir6 + (size_t)r * 6 + c - 3;
                    *dst = acc ? *dst + v : v;
                });
            }
            __syncthreads();                               // slots read before the next basis overwrites them
        }
    }
    const bool drained = drain_mma(mma_out, &S.mbar, pend);   // as in the forward kernel
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
    if (!ok && tid == 0) atomicOr(status, drained ? 1 : 3);
}

// ------------------------------------------------------------ backward, NG tiles per CTA
// The same pass with NG tiles in flight per CTA: NG groups of 4 warps, each
// with its own tile buffers, tensor-memory columns, mbarrier and named
// barrier, sharing one copy of the weight tiles. The second and third MMAs
// take their A operand from tensor memory, which keeps one tile in 2F
// columns: per group X = [0, F) and Y = [F, 2F),
//   MMA1:  D1 -> X, D4 -> Y
//   epi 1: p = SiLU'(a)(e'W1) as BF16 -> X[0, F/2); SiLU(a) as BF16 -> Y[0, F/2)
//   MMA2:  D2 = SiLU W2 as two N = F/2 halves -> X[F/2, F), Y[F/2, F)
//   epi 2: g as BF16 -> Y[0, F/2)
//   MMA3:  D3 = g W2^T as two halves -> X[F/2, F), Y[F/2, F)
//   epi 3: sum_k D3_k p_k
// (each epilogue writes a BF16 chunk only into columns it has already read).
template <int F>
struct alignas(16) BwdGroup {
    unsigned char a14[2 * kT * kKP * 2];  // basis | basis derivative; then the tile's vector and scalar slots
    float G[kT * F];                       // gathered BF16 rows of u_j | mbar_j, then the FP32 ubar messages
    uint64_t mbar;
    uint64_t pad;
};

template <int F, int NG>
struct BwdGSmem {
    unsigned char w1t[F * kKP * 2];       // B[n][k] = W1[k][n]
    unsigned char w2t[F * F * 2];         // B[n][k] = W2[k][n]
    unsigned char w2n[F * F * 2];         // B[n][k] = W2[n][k]
    float b1[F], b2[F];
    BwdGroup<F> grp[NG];
    uint32_t taddr;
};

// Named barrier of one 128-thread group (ids 1 .. NG; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "n"(kT) : "memory");
}
__device__ __forceinline__ bool group_sync_and(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t"
        ".reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t"
        "}"
        : "=r"(r) : "r"((uint32_t)v), "r"(id), "n"(kT) : "memory");
    return r != 0;
}

__device__ __forceinline__ void unpack_bf16x16(const uint32_t* w, float* v) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);
        v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}

template <int F, int NV, int NG, int KC, bool L0>
__global__ void __launch_bounds__(kT * NG, 2) k_edge_bwd_grp(PotArgs a, int K, int* status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    BwdGSmem<F, NG>& S = *reinterpret_cast<BwdGSmem<F, NG>*>(smraw);
    constexpr int H = F / 2;
    const int g = threadIdx.x / kT;                    // this thread's group
    const int tid = threadIdx.x & (kT - 1), warp = tid >> 5;
    const int bar = 1 + g;
    BwdGroup<F>& T = S.grp[g];
    static_assert(scal_slot_offset<F>() + sizeof(ScalSlots<NV>) <= sizeof(T.a14), "slots must fit the basis tiles");
    static_assert(H % 16 == 0, "half the features must be whole 16-column chunks");
    VecSlots<F>* vs = reinterpret_cast<VecSlots<F>*>(T.a14);
    ScalSlots<NV>* ss = reinterpret_cast<ScalSlots<NV>*>(T.a14 + scal_slot_offset<F>());
    unsigned char* const a1 = T.a14;
    unsigned char* const a4 = T.a14 + kT * kKP * 2;
    const int l = a.layer;
    const long long E = min((long long)a.row_ptr[a.n_atoms], a.e_cap);
    const long long n_tiles = (E + kT - 1) / kT;
    constexpr bool need_ubar = !L0;

    {
        const uint4* src = reinterpret_cast<const uint4*>(a.wt + (size_t)l * a.wt_layer_bytes);
        uint4* d1 = reinterpret_cast<uint4*>(S.w1t);
        uint4* d2 = reinterpret_cast<uint4*>(S.w2t);
        uint4* d3 = reinterpret_cast<uint4*>(S.w2n);
        for (int t = threadIdx.x; t < F * kKP * 2 / 16; t += kT * NG) d1[t] = src[t];
        src += F * kKP * 2 / 16;
        for (int t = threadIdx.x; t < F * F * 2 / 16; t += kT * NG) d2[t] = src[t];
        src += F * F * 2 / 16;
        for (int t = threadIdx.x; t < F * F * 2 / 16; t += kT * NG) d3[t] = src[t];
    }
    for (int t = threadIdx.x; t < F; t += kT * NG) {
        S.b1[t] = __ldg(a.P + a.off.b1[l] + t);
        S.b2[t] = __ldg(a.P + a.off.b2[l] + t);
    }
    if (tid == 0) mbar_init(&T.mbar, 1);
    if (threadIdx.x < 32) tmem_alloc(&S.taddr, NG * 2 * F);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t tX = S.taddr + g * 2 * F, tY = tX + F;
    const uint32_t idesc = idesc_bf16_f32(128, F), idesc_h = idesc_bf16_f32(128, H);
    const uint32_t sA1 = smem_u32(a1), sA4 = smem_u32(a4);
    const uint32_t sW1T = smem_u32(S.w1t), sW2T = smem_u32(S.w2t), sW2N = smem_u32(S.w2n);
    uint32_t phase = 0;
    bool ok = true;
    bool mma_out = false;                                  // thread 0: a commit not yet seen complete
    uint32_t pend = 0;                                     // ... and the parity it completes

    const int cw = a.carry_w;
    const long long first = (long long)blockIdx.x * NG + g, step = (long long)gridDim.x * NG;
    EdgeIn nx;
    load_idx(a, first * kT + tid, E, nx);
    load_pos(a, nx);
    for (long long tile = first; tile < n_tiles && ok; tile += step) {
        const long long tb = tile * kT, te = min(tb + kT, E);
        int prev_row = -1, next_row = -1;                  // read by the merges at the end of the tile
        if (tid < F + NV) {
            if (tb > 0) prev_row = __ldg(a.recv + tb - 1);
            if (te < E) next_row = __ldg(a.recv + te);
        }
        const EdgeIn ex = nx;
        const bool valid = ex.j >= 0;
        const int j = valid ? ex.j : 0;
        const int row = valid ? ex.i : -1;
        if (valid)
            fill_empty_rows<F>(ex.rp, row, tb + tid == E - 1, a.n_atoms, need_ubar ? a.msg_out : nullptr,
                               [&](int r) { zero_force_row<NV>(a, r); });
        load_idx(a, (tile + step) * kT + tid, E, nx);      // this group's next tile's indices
        gather_rows<F>(T.G, reinterpret_cast<const float*>(a.um), j, tid);
        cp_async_commit();
        if (valid) {                                       // the receiving atom's rows, read in the second epilogue
            prefetch_row_l1<F>(a.u + (size_t)row * F);
            prefetch_row_l1<F>(a.mbar + (size_t)row * F);
        }
        float fc = 0.f, dfc = 0.f, d = 1.f, rx = 0.f, ry = 0.f, rz = 0.f;
        {
            float eb[kKP], db[kKP];
            if (valid) {
                const uint4 qi = ex.qi, qj = ex.qj;
                float3 r = edge_vec(qi, qj, a.frame[qi.w].qscale);
                float r2 = r.x * r.x + r.y * r.y + r.z * r.z;
                float inv = rsqrtf(r2);
                d = r2 * inv;
                rx = r.x * inv; ry = r.y * inv; rz = r.z * inv;
                basis16<KC>(d, inv, K, a.pi_over_rc, a.bessel_pref, eb, db, fc, dfc);
            } else {
#pragma unroll
                for (int k = 0; k < kKP; ++k) { eb[k] = 0.f; db[k] = 0.f; }
            }
            st_row8(a1, tid, 0, kKP, eb);
            st_row8(a1, tid, 8, kKP, eb + 8);
            st_row8(a4, tid, 0, kKP, db);
            st_row8(a4, tid, 8, kKP, db + 8);
        }
        fence_proxy_async();
        fence_before_sync();
        group_sync(bar);
        fence_after_sync();
        if (tid == 0) {
            mma_bf16(tX, make_desc(sA1, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
            mma_bf16(tY, make_desc(sA4, 128, kKP * 16), make_desc(sW1T, 128, kKP * 16), idesc, 0);
            mma_commit(&T.mbar);
            mma_out = true;
            pend = phase;
        }
        load_pos(a, nx);                                   // next tile's positions
        ok = mbar_wait(&T.mbar, phase, kWaitIter);
        if (tid == 0 && ok) mma_out = false;
        phase ^= 1;
        fence_after_sync();
        float se;
        if constexpr (!need_ubar) {
            // Layer 0 (u independent of the positions), as in the one-tile kernel:
            //   epi 1: q = dfc SiLU(a) + fc SiLU'(a)(e'W1) as BF16 -> X[0, F/2)
            //   epi 2: g as BF16 -> Y[0, F/2)
            //   MMA3:  D3 = g W2^T as two halves -> X[F/2, F), Y[F/2, F)
            //   epi 3: sum_k D3_k q_k + dfc (g . b2)
            const f2::f32x2 fc2 = f2::splat(fc), dfc2 = f2::splat(dfc);
#pragma unroll
            for (int c = 0; c < F; c += 16) {
                float v[16], tv[16];
                tmem_ld16x2(tX + lane_base + c, v, tY + lane_base + c, tv);
                uint32_t pq[8];
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const f2::f32x2 x = f2::add(f2::pack(v[q], v[q + 1]), *reinterpret_cast<const f2::f32x2*>(S.b1 + c + q));
                    const f2::f32x2 t = tanh_half(x);
                    const f2::f32x2 sg = f2::fma(kHalf2, t, kHalf2), sgc = f2::fma(kMinusHalf2, t, kHalf2);
                    const f2::f32x2 y = f2::mul(x, sg);
                    const f2::f32x2 pd = f2::mul(f2::pack(tv[q], tv[q + 1]), f2::fma(y, sgc, sg));
                    const f2::f32x2 qv = f2::fma(dfc2, y, f2::mul(fc2, pd));
                    pq[q / 2] = pack_bf16(f2::lo(qv), f2::hi(qv));
                }
                tmem_st8(tX + lane_base + c / 2, pq);
            }
            cp_async_wait();                               // the warp's u_j | mbar_j rows are in G
            __syncwarp();
            f2::f32x2 gb22 = 0ull;
            {
                const int i = valid ? row : 0;
                const float* ui = a.u + (size_t)i * F;
                const float* mi = a.mbar + (size_t)i * F;
#pragma unroll
                for (int c = 0; c < F; c += 16) {
                    uint4 w[4];                            // BF16 u_j (w[0], w[1]) and mbar_j (w[2], w[3])
#pragma unroll
                    for (int k = 0; k < 4; ++k) w[k] = *reinterpret_cast<const uint4*>(T.G + prow<F>(tid, c + 4 * k));
                    uint32_t pg[8];
#pragma unroll
                    for (int q = 0; q < 16; q += 4) {
                        const float4 ui4 = __ldg(reinterpret_cast<const float4*>(ui + c + q));
                        const float4 mi4 = __ldg(reinterpret_cast<const float4*>(mi + c + q));
                        const uint32_t u01 = q < 8 ? (q == 0 ? w[0].x : w[0].z) : (q == 8 ? w[1].x : w[1].z);
                        const uint32_t u23 = q < 8 ? (q == 0 ? w[0].y : w[0].w) : (q == 8 ? w[1].y : w[1].w);
                        const uint32_t m01 = q < 8 ? (q == 0 ? w[2].x : w[2].z) : (q == 8 ? w[3].x : w[3].z);
                        const uint32_t m23 = q < 8 ? (q == 0 ? w[2].y : w[2].w) : (q == 8 ? w[3].y : w[3].w);
                        const f2::f32x2 uj01 = f2::from_bf16x2(u01), uj23 = f2::from_bf16x2(u23);
                        const f2::f32x2 mj01 = f2::from_bf16x2(m01), mj23 = f2::from_bf16x2(m23);
                        const f2::f32x2* b2 = reinterpret_cast<const f2::f32x2*>(S.b2 + c + q);
                        const f2::f32x2 g01 = f2::fma(f2::pack(mi4.x, mi4.y), uj01, f2::mul(mj01, f2::pack(ui4.x, ui4.y)));
                        const f2::f32x2 g23 = f2::fma(f2::pack(mi4.z, mi4.w), uj23, f2::mul(mj23, f2::pack(ui4.z, ui4.w)));
                        gb22 = f2::fma(g01, b2[0], gb22);
                        gb22 = f2::fma(g23, b2[1], gb22);
                        pg[q / 2] = pack_bf16(f2::lo(g01), f2::hi(g01));
                        pg[q / 2 + 1] = pack_bf16(f2::lo(g23), f2::hi(g23));
                    }
                    tmem_st8(tY + lane_base + c / 2, pg);  // over e'W1 (read by epilogue 1)
                }
            }
            tmem_st_wait();
            fence_before_sync();
            ok = group_sync_and(bar, ok);
            fence_after_sync();
            if (tid == 0 && ok) {
#pragma unroll
                for (int kk = 0; kk < F / 16; ++kk) {
                    mma_bf16_ta(tX + H, tY + kk * 8, make_desc(sW2N + kk * 256, 128, F * 16), idesc_h, kk > 0);
                    mma_bf16_ta(tY + H, tY + kk * 8, make_desc(sW2N + F * F + kk * 256, 128, F * 16), idesc_h, kk > 0);
                }
                mma_commit(&T.mbar);
                mma_out = true;
                pend = phase;
            }
            ok = ok && mbar_wait(&T.mbar, phase, kWaitIter);
            if (tid == 0 && ok) mma_out = false;
            phase ^= 1;
            fence_after_sync();
            f2::f32x2 s22 = 0ull;
#pragma unroll
            for (int c = 0; c < F; c += 16) {
                float ab[16];
                uint32_t pw[8];
                tmem_ld16_8((c < H ? tX : tY) + H + (c % H) + lane_base, ab, tX + lane_base + c / 2, pw);
#pragma unroll
                for (int q = 0; q < 16; q += 2) s22 = f2::fma(f2::pack(ab[q], ab[q + 1]), f2::from_bf16x2(pw[q / 2]), s22);
            }
            se = __fmaf_rn(dfc, f2::lo(gb22) + f2::hi(gb22), f2::lo(s22) + f2::hi(s22));
        } else {
            // epilogue 1: p = SiLU'(a)(e'W1) -> X[0, F/2), SiLU(a) -> Y[0, F/2), both BF16
#pragma unroll
            for (int c = 0; c < F; c += 16) {
                float v[16], tv[16];
                tmem_ld16x2(tX + lane_base + c, v, tY + lane_base + c, tv);
                uint32_t ps[8], pp[8];
#pragma unroll
                for (int q = 0; q < 16; q += 2) {              // two features per packed FP32 operation
                    const f2::f32x2 x = f2::add(f2::pack(v[q], v[q + 1]), *reinterpret_cast<const f2::f32x2*>(S.b1 + c + q));
                    const f2::f32x2 t = tanh_half(x);            // sigmoid(x) = (1 + tanh(x / 2)) / 2
                    const f2::f32x2 sg = f2::fma(kHalf2, t, kHalf2), sgc = f2::fma(kMinusHalf2, t, kHalf2);
                    const f2::f32x2 y = f2::mul(x, sg);          // SiLU
                    const f2::f32x2 pd = f2::mul(f2::pack(tv[q], tv[q + 1]), f2::fma(y, sgc, sg));   // SiLU' (e'W1)
                    ps[q / 2] = pack_bf16(f2::lo(y), f2::hi(y));
                    pp[q / 2] = pack_bf16(f2::lo(pd), f2::hi(pd));
                }
                tmem_st8(tY + lane_base + c / 2, ps);
                tmem_st8(tX + lane_base + c / 2, pp);
            }
            tmem_st_wait();
            fence_before_sync();
            ok = group_sync_and(bar, ok);
            fence_after_sync();
            if (tid == 0 && ok) {
#pragma unroll
                for (int kk = 0; kk < F / 16; ++kk) {
                    mma_bf16_ta(tX + H, tY + kk * 8, make_desc(sW2T + kk * 256, 128, F * 16), idesc_h, kk > 0);
                    mma_bf16_ta(tY + H, tY + kk * 8, make_desc(sW2T + F * F + kk * 256, 128, F * 16), idesc_h, kk > 0);
                }
                mma_commit(&T.mbar);
                mma_out = true;
                pend = phase;
            }
            ok = ok && mbar_wait(&T.mbar, phase, kWaitIter);
            if (tid == 0 && ok) mma_out = false;
            phase ^= 1;
            fence_after_sync();
            cp_async_wait();                                   // the warp's u_j | mbar_j rows are in G
            __syncwarp();
            f2::f32x2 gphi2 = 0ull;                            // (+0, +0)
            {
                const int i = valid ? row : 0;
                const float* ui = a.u + (size_t)i * F;
                const float* mi = a.mbar + (size_t)i * F;
#pragma unroll
                for (int c = 0; c < F; c += 16) {
                    float v[16];
                    tmem_ld16((c < H ? tX : tY) + H + (c % H) + lane_base, v);
                    uint4 w[4];                                // BF16 u_j (w[0], w[1]) and mbar_j (w[2], w[3])
#pragma unroll
                    for (int k = 0; k < 4; ++k) w[k] = *reinterpret_cast<const uint4*>(T.G + prow<F>(tid, c + 4 * k));
                    uint32_t pg[8];
                    const f2::f32x2 fc2 = f2::splat(fc);
#pragma unroll
                    for (int q = 0; q < 16; q += 4) {
                        const float4 ui4 = __ldg(reinterpret_cast<const float4*>(ui + c + q));
                        const float4 mi4 = __ldg(reinterpret_cast<const float4*>(mi + c + q));
                        const uint32_t u01 = q < 8 ? (q == 0 ? w[0].x : w[0].z) : (q == 8 ? w[1].x : w[1].z);
                        const uint32_t u23 = q < 8 ? (q == 0 ? w[0].y : w[0].w) : (q == 8 ? w[1].y : w[1].w);
                        const uint32_t m01 = q < 8 ? (q == 0 ? w[2].x : w[2].z) : (q == 8 ? w[3].x : w[3].z);
                        const uint32_t m23 = q < 8 ? (q == 0 ? w[2].y : w[2].w) : (q == 8 ? w[3].y : w[3].w);
                        const f2::f32x2 uj01 = f2::from_bf16x2(u01), uj23 = f2::from_bf16x2(u23);
                        const f2::f32x2 mj01 = f2::from_bf16x2(m01), mj23 = f2::from_bf16x2(m23);
                        const f2::f32x2* b2 = reinterpret_cast<const f2::f32x2*>(S.b2 + c + q);
                        const f2::f32x2 ph01 = f2::add(f2::pack(v[q], v[q + 1]), b2[0]);
                        const f2::f32x2 ph23 = f2::add(f2::pack(v[q + 2], v[q + 3]), b2[1]);
                        // g = mbar_i u_j + mbar_j u_i
                        const f2::f32x2 g01 = f2::fma(f2::pack(mi4.x, mi4.y), uj01, f2::mul(mj01, f2::pack(ui4.x, ui4.y)));
                        const f2::f32x2 g23 = f2::fma(f2::pack(mi4.z, mi4.w), uj23, f2::mul(mj23, f2::pack(ui4.z, ui4.w)));
                        gphi2 = f2::fma(g01, ph01, gphi2);
                        gphi2 = f2::fma(g23, ph23, gphi2);
                        pg[q / 2] = pack_bf16(f2::lo(g01), f2::hi(g01));
                        pg[q / 2 + 1] = pack_bf16(f2::lo(g23), f2::hi(g23));
                        // the message replaces the chunk (read above into w) of this thread's row
                        const f2::f32x2 o01 = f2::mul(f2::mul(fc2, ph01), mj01), o23 = f2::mul(f2::mul(fc2, ph23), mj23);
                        *reinterpret_cast<float4*>(T.G + prow<F>(tid, c + q)) =
                            make_float4(f2::lo(o01), f2::hi(o01), f2::lo(o23), f2::hi(o23));
                    }
                    tmem_st8(tY + lane_base + c / 2, pg);     // over SiLU (read by the completed MMA2)
                }
            }
            tmem_st_wait();
            fence_before_sync();
            ok = group_sync_and(bar, ok);
            fence_after_sync();
            if (tid == 0 && ok) {
#pragma unroll
                for (int kk = 0; kk < F / 16; ++kk) {
                    mma_bf16_ta(tX + H, tY + kk * 8, make_desc(sW2N + kk * 256, 128, F * 16), idesc_h, kk > 0);
                    mma_bf16_ta(tY + H, tY + kk * 8, make_desc(sW2N + F * F + kk * 256, 128, F * 16), idesc_h, kk > 0);
                }
                mma_commit(&T.mbar);
                mma_out = true;
                pend = phase;
            }
            ok = ok && mbar_wait(&T.mbar, phase, kWaitIter);
            if (tid == 0 && ok) mma_out = false;
            phase ^= 1;
            fence_after_sync();
            f2::f32x2 s22 = 0ull;
#pragma unroll
            for (int c = 0; c < F; c += 16) {
                float ab[16];
                uint32_t pw[8];
                tmem_ld16_8((c < H ? tX : tY) + H + (c % H) + lane_base, ab, tX + lane_base + c / 2, pw);
#pragma unroll
                for (int q = 0; q < 16; q += 2) s22 = f2::fma(f2::pack(ab[q], ab[q + 1]), f2::from_bf16x2(pw[q / 2]), s22);
            }
            const float gphi = f2::lo(gphi2) + f2::hi(gphi2), s2 = f2::lo(s22) + f2::hi(s22);
            se = dfc * gphi + fc * s2;
        }
        if (L0 && valid) {
            float dphi;
            (void)rep_phi(d, a.rep_a, a.rep_inv_rho, a.rep_rc, a.rep_pi_over_rc, &dphi);
            se += dphi;
        }
        {
            float val[NV];
            val[0] = se * rx; val[1] = se * ry; val[2] = se * rz;
            if constexpr (NV == 9) {
                float hv = -0.5f * se * d;
                val[3] = hv * rx * rx; val[4] = hv * ry * ry; val[5] = hv * rz * rz;
                val[6] = hv * rx * ry; val[7] = hv * rx * rz; val[8] = hv * ry * rz;
            }
            warp_scal_segments<NV>(val, row, ss, tid);
        }
        fence_before_sync();
        ok = group_sync_and(bar, ok);
        if (need_ubar) warp_vec_segments<F>(T.G, row, vs, a.msg_out, 0, tid);
        group_sync(bar);
        const TileCtx tc{prev_row, next_row, a.carry + 2 * tile * cw, a.carry + (2 * tile + 1) * cw};
        if (need_ubar && tid < F) {
            merge_tile_vec<F>(vs, tid, tc, a.msg_out);
        } else if (tid >= F && tid < F + NV) {
            float* force = a.force;
            float* vir6 = a.vir6;
            const int n = a.n_atoms, acc = a.accumulate;
            merge_tile_scal<NV, F>(ss, tid - F, tc, [=](int r, int c, float v) {
                float* dst = c < 3 ? force + (size_t)c * n + r : vir6 + (size_t)r * 6 + c - 3;
                *dst = acc ? *dst + v : v;
            });
        }
        group_sync(bar);                                   // slots read before the next basis overwrites them
    }
    const bool drained = drain_mma(mma_out, &T.mbar, pend);   // each group's issuing thread, as above
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(S.taddr, NG * 2 * F);
    if (!ok && tid == 0) atomicOr(status, drained ? 1 : 3);
}

// CTAs of a kernel that fit on one SM: shared memory (1 KB reserved per
// CTA), the 512 tensor-memory columns, registers (allocated per warp in
// multiples of 8 per thread) and threads.
template <class Kern>
int ctas_per_sm_limit(Kern kern, int smem, int tmem_cols, int threads) {
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        smem_sm = 233472;
    }
    int regs = 0;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess) regs = fa.numRegs;
    else cudaGetLastError();
    const int by_regs = regs > 0 ? 65536 / (((regs + 7) / 8 * 8) * threads) : 64;
    return std::max(1, std::min({smem_sm / (smem + 1024), 512 / tmem_cols, by_regs, 2048 / threads}));
}

// SM count and CTAs per SM that fit, per kernel and device (computed at the
// first launch on each device).
struct PersistLimits {
    int sms = 0, per_sm = 0;
};
std::mutex g_limits_mu;
std::map<std::pair<const void*, int>, PersistLimits> g_limits;

template <class Kern>
PersistLimits persist_limits(Kern kern, int smem, int tmem_cols, int threads) {
    int dev = 0;
    cudaGetDevice(&dev);
    const std::pair<const void*, int> key{(const void*)kern, dev};
    std::lock_guard<std::mutex> lock(g_limits_mu);
    auto it = g_limits.find(key);
    if (it != g_limits.end()) return it->second;
    smem_opt_in((const void*)kern, smem);
    PersistLimits lim;
    if (cudaDeviceGetAttribute(&lim.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        lim.sms = 1;
    }
    lim.per_sm = ctas_per_sm_limit(kern, smem, tmem_cols, threads);
    g_limits[key] = lim;
    return lim;
}

// Persistent launch: SMs x CTAs per SM, bounded as above and by the tuner's
// choice; never more CTAs than needed for the tiles the pair capacity can
// hold (tiles_per_cta tiles in flight per CTA).
template <class Kern>
void launch_persistent(Kern kern, int smem, int tmem_cols, int threads, int tiles_per_cta, const PotArgs& a, int K,
                       int* status, cudaStream_t s) {
    const PersistLimits lim = persist_limits(kern, smem, tmem_cols, threads);
    const int per_sm = a.ctas_per_sm > 0 ? std::min(a.ctas_per_sm, lim.per_sm) : lim.per_sm;
    const long long tiles = (a.e_cap + kT - 1) / kT;
    const long long grid = std::min<long long>((tiles + tiles_per_cta - 1) / tiles_per_cta, (long long)lim.sms * per_sm);
    if (grid > 0) kern<<<(int)grid, threads, smem, s>>>(a, K, status);
}

// Tiles in flight per CTA of the grouped backward kernel (k_edge_bwd_grp).
constexpr int kBwdGroups = 2;

// The radial-function count compiled into the kernels of each width (the
// big model: F = 64, K = 16; the small one: F = 32, K = 8); other counts use
// the kernels that take K at run time.
template <int F>
constexpr int kSpecK = F == 64 ? 16 : 8;

template <int F, int KC>
void go_fwd(const PotArgs& a, int K, int* status, cudaStream_t s) {
    launch_persistent(k_edge_fwd_bf16<F, KC>, (int)sizeof(FwdSmem<F>), 2 * F, kT, 1, a, K, status, s);
    if (a.fused_fixup) return;                         // the per-atom kernel sums the split rows
    k_tile_fixup<F><<<fixup_blocks(a.e_cap), 256, 0, s>>>(a.n_atoms, a.row_ptr, a.recv, a.e_cap, a.carry,
                                                          a.carry_w, a.msg_out, a.layer == 0 ? 1 : 0, 0, a.erep,
                                                          nullptr, nullptr, 0, a.check);
}

template <int F, int NV, int KC, bool L0>
void go_bwd_layer(const PotArgs& a, int K, int* status, cudaStream_t s) {
    const int tiles = a.bwd_tiles > 0 ? a.bwd_tiles : bf16_default_bwd_tiles(F);
    if (tiles == 2)
        launch_persistent(k_edge_bwd_grp<F, NV, kBwdGroups, KC, L0>, (int)sizeof(BwdGSmem<F, kBwdGroups>),
                          kBwdGroups * 2 * F, kT * kBwdGroups, kBwdGroups, a, K, status, s);
    else
        launch_persistent(k_edge_bwd_bf16<F, NV, KC, L0>, (int)sizeof(BwdSmem<F, NV>), 2 * F, kT, 1, a, K, status, s);
}

template <int F, int NV, int KC>
void go_bwd(const PotArgs& a, int K, int* status, cudaStream_t s) {
    if (a.layer == 0) go_bwd_layer<F, NV, KC, true>(a, K, status, s);
    else go_bwd_layer<F, NV, KC, false>(a, K, status, s);
    if (a.fold_fixup && a.layer == 0 && !a.accumulate && NV == 3) return;   // the integrator sums the split rows
    k_tile_fixup<F><<<fixup_blocks(a.e_cap), 256, 0, s>>>(a.n_atoms, a.row_ptr, a.recv, a.e_cap, a.carry,
                                                          a.carry_w, a.layer > 0 ? a.msg_out : nullptr, NV, 1,
                                                          nullptr, a.force, a.vir6, a.accumulate, a.check);
}

template <int F>
void fwd_k(const PotArgs& a, int K, int* status, cudaStream_t s) {
    if (K == kSpecK<F>) go_fwd<F, kSpecK<F>>(a, K, status, s);
    else go_fwd<F, 0>(a, K, status, s);
}

template <int F, int NV>
void bwd_k(const PotArgs& a, int K, int* status, cudaStream_t s) {
    if (K == kSpecK<F>) go_bwd<F, NV, kSpecK<F>>(a, K, status, s);
    else go_bwd<F, NV, 0>(a, K, status, s);
}

// Self-test of the bounded completion waits, issuing no MMA: warp 0 takes 32
// tensor-memory columns, the mbarrier expects one arrival, thread 0 arrives
// only if `arrive` is set, and every thread waits through the same bounded
// wait as the force kernels, at most `polls` polls. The columns are freed
// either way, and a wait that gave up sets status bit 0, as in those kernels.
__global__ void __launch_bounds__(kT) k_wait_selftest(int arrive, uint32_t polls, int* status) {
    __shared__ uint64_t mbar;
    __shared__ uint32_t taddr;
    const int tid = threadIdx.x;
    if (tid == 0) mbar_init(&mbar, 1);
    if (tid < 32) tmem_alloc(&taddr, 32);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (arrive && tid == 0) mbar_arrive(&mbar);
    const bool ok = mbar_wait(&mbar, 0, polls);
    fence_before_sync();
    __syncthreads();
    if (tid < 32) tmem_dealloc(taddr, 32);
    if (!ok && (tid & 31) == 0) atomicOr(status, 1);
}

}  // namespace

void launch_wait_selftest(int arrive, unsigned int polls, int* status, cudaStream_t s) {
    k_wait_selftest<<<1, kT, 0, s>>>(arrive, polls, status);
    count_launch();
}

void launch_edge_fwd_bf16(const PotArgs& a, int F, int K, int* status, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    if (F == 64) fwd_k<64>(a, K, status, s);
    else fwd_k<32>(a, K, status, s);
    count_launch(a.fused_fixup ? 1 : 2);
}

void launch_edge_bwd_bf16(const PotArgs& a, int F, int K, int* status, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    if (a.virial) {
        if (F == 64) bwd_k<64, 9>(a, K, status, s);
        else bwd_k<32, 9>(a, K, status, s);
    } else {
        if (F == 64) bwd_k<64, 3>(a, K, status, s);
        else bwd_k<32, 3>(a, K, status, s);
    }
    count_launch(a.fold_fixup && a.layer == 0 && !a.accumulate && !a.virial ? 1 : 2);
}

// The backward kernel's tiles in flight per CTA unless the tuner chooses:
// two at F = 64 (two groups of 4 warps share one copy of the weights), one
// at F = 32, where the one-tile kernel fits 5 CTAs of 4 warps per SM
// against 2 of 8 (28.6 vs 31.6 us measured on 12,288-atom water).
int bf16_default_bwd_tiles(int F) { return F == 64 ? 2 : 1; }

int bf16_max_ctas_per_sm(int F, bool bwd, int tiles) {
    if (bwd) {
        constexpr int G = kBwdGroups;
        if (tiles <= 0) tiles = bf16_default_bwd_tiles(F);
        // the fewer of the two layer variants
        if (tiles == 2)
            return F == 64 ? std::min(ctas_per_sm_limit(k_edge_bwd_grp<64, 3, G, kSpecK<64>, false>,
                                                        (int)sizeof(BwdGSmem<64, G>), G * 128, kT * G),
                                      ctas_per_sm_limit(k_edge_bwd_grp<64, 3, G, kSpecK<64>, true>,
                                                        (int)sizeof(BwdGSmem<64, G>), G * 128, kT * G))
                           : std::min(ctas_per_sm_limit(k_edge_bwd_grp<32, 3, G, kSpecK<32>, false>,
                                                        (int)sizeof(BwdGSmem<32, G>), G * 64, kT * G),
                                      ctas_per_sm_limit(k_edge_bwd_grp<32, 3, G, kSpecK<32>, true>,
                                                        (int)sizeof(BwdGSmem<32, G>), G * 64, kT * G));
        return F == 64 ? std::min(ctas_per_sm_limit(k_edge_bwd_bf16<64, 3, kSpecK<64>, false>,
                                                    (int)sizeof(BwdSmem<64, 3>), 128, kT),
                                  ctas_per_sm_limit(k_edge_bwd_bf16<64, 3, kSpecK<64>, true>,
                                                    (int)sizeof(BwdSmem<64, 3>), 128, kT))
                       : std::min(ctas_per_sm_limit(k_edge_bwd_bf16<32, 3, kSpecK<32>, false>,
                                                    (int)sizeof(BwdSmem<32, 3>), 64, kT),
                                  ctas_per_sm_limit(k_edge_bwd_bf16<32, 3, kSpecK<32>, true>,
                                                    (int)sizeof(BwdSmem<32, 3>), 64, kT));
    }
    return F == 64 ? ctas_per_sm_limit(k_edge_fwd_bf16<64, kSpecK<64>>, (int)sizeof(FwdSmem<64>), 128, kT)
                   : ctas_per_sm_limit(k_edge_fwd_bf16<32, kSpecK<32>>, (int)sizeof(FwdSmem<32>), 64, kT);
}

size_t bf16_weight_tile_bytes(int F) {
    // per layer: W1^T [F][16], W2^T [F][F], W2 [F][F], each BF16 in the K-major tile layout
    return (size_t)F * kKP * 2 + 2 * (size_t)F * F * 2;
}

}  // namespace dmts
