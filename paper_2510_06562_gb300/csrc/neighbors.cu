// Fixed-point positions, cell lists and neighbour CSR.
//
// The pair set is {(i, j) : j != i, same system, |r_ij|^2 < rc^2} with r_ij
// the minimum-image difference evaluated in FP64 with every operation rounded
// separately. GB300 runs FP64 at a small fraction of its FP32 rate, so each
// candidate is first classified in FP32 from 32-bit fixed-point coordinates
// (the wrapped integer difference is the minimum image); only candidates in
// a thin band around rc^2, where FP32 rounding could flip the decision, are
// decided by the exact FP64 expression.
//
// Fresh lists (skin 0) use cells of fixed capacity: one kernel puts every
// atom into the next free slot of its cell (an atomic counter per cell), the
// row build reads the 27 cells around each atom at fixed strides and sorts
// each row by j (so the list does not depend on the slot order) and adds
// its pair count to per-block and per-chunk sums, and the compaction finds
// each row's offset from those sums, writes the CSR arrays and clears the
// cell counters for the next build.
//
// Verlet-skin mode keeps, per model, candidate rows of every j within
// rc + skin at the positions x_ref of the last rebuild. While no atom has
// moved by skin / 2 or more since then, every pair now inside rc was inside
// rc + skin at the rebuild (|r_now| >= |r_ref| - |dx_i| - |dx_j|), so the
// exact test applied to the candidate rows yields the same pair set as a
// fresh build. The rebuild decision is taken on the device: the rebuild
// kernels stay in the stream (and in captured graphs) and return at once
// when their gate is clear.
#include <algorithm>

#include "internal.cuh"

namespace dmts {

// ------------------------------------------------------------ frames
// Non-periodic systems: origin = lower corner of the bounding box, Q = the
// smallest power of two >= 2 (extent + 2 rc_max + 1) so that every in-cutoff
// difference stays far below Q/2. Periodic systems: origin 0, Q = L.
__global__ void k_frames(int n_sys, const int* __restrict__ off, const double* __restrict__ x,
                         int n, const double* __restrict__ box, double rc_max,
                         Frame* __restrict__ frame) {
    int s = blockIdx.x;
    if (s >= n_sys) return;
    double L = box[s];
    if (L > 0.0) {
        if (threadIdx.x == 0) {
            Frame f;
            f.ox = f.oy = f.oz = 0.0;
            f.inv = 4294967296.0 / L;
            f.qscale = (float)(L / 4294967296.0);
            f.pad = 0.f;
            frame[s] = f;
        }
        return;
    }
    __shared__ double smin[3][32], smax[3][32];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            double v = x[(size_t)c * n + i];
            lo[c] = fmin(lo[c], v);
            hi[c] = fmax(hi[c], v);
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int c = 0; c < 3; ++c) { smin[c][w] = lo[c]; smax[c][w] = hi[c]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        double ext = 0.0, o3[3];
        for (int c = 0; c < 3; ++c) {
            double a = 1e300, b = -1e300;
            for (int k = 0; k < nw; ++k) { a = fmin(a, smin[c][k]); b = fmax(b, smax[c][k]); }
            if (off[s + 1] == off[s]) { a = 0.0; b = 0.0; }
            o3[c] = a;
            ext = fmax(ext, b - a);
        }
        double need = 2.0 * (ext + 2.0 * rc_max + 1.0);
        double Q = 1.0;
        while (Q < need) Q *= 2.0;
        Frame f;
        f.ox = o3[0]; f.oy = o3[1]; f.oz = o3[2];
        f.inv = 4294967296.0 / Q;
        f.qscale = (float)(Q / 4294967296.0);
        f.pad = 0.f;
        frame[s] = f;
    }
}

void launch_frames(int n_sys, const int* atom_offset, const double* x, int n_atoms,
                   const double* box, double rc_max, Frame* frame, cudaStream_t s) {
    k_frames<<<n_sys, 256, 0, s>>>(n_sys, atom_offset, x, n_atoms, box, rc_max, frame);
    count_launch();
}

__device__ __forceinline__ unsigned int to_fixed(double v, double o, double inv) {
    double t = floor((v - o) * inv);
    long long k = (long long)t;
    return (unsigned int)(k & 0xffffffffll);
}

__global__ void k_quantize(int n, const double* __restrict__ x, const int* __restrict__ sys,
                           const Frame* __restrict__ frame, uint4* __restrict__ q) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = sys[i];
    Frame f = frame[s];
    uint4 r;
    r.x = to_fixed(x[i], f.ox, f.inv);
    r.y = to_fixed(x[(size_t)n + i], f.oy, f.inv);
    r.z = to_fixed(x[2 * (size_t)n + i], f.oz, f.inv);
    r.w = (unsigned int)s;
    q[i] = r;
}

void launch_quantize(int n_atoms, const double* x, const int* sys_of_atom, const Frame* frame,
                     uint4* q, cudaStream_t s) {
    if (n_atoms == 0) return;
    k_quantize<<<(n_atoms + 255) / 256, 256, 0, s>>>(n_atoms, x, sys_of_atom, frame, q);
    count_launch();
}

// ------------------------------------------------------------ cell list
__device__ __forceinline__ bool gated_off(const int* gate) { return gate && *gate == 0; }

__global__ void k_cell_clear(int n, int* __restrict__ count, const int* gate) {
    if (gated_off(gate)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) count[i] = 0;
}

__global__ void k_cell_count(int n, const uint4* __restrict__ q, int nc, int* __restrict__ count,
                             int* __restrict__ atom_cell, int* __restrict__ slot, const int* gate) {
    if (gated_off(gate)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 p = q[i];
    int c = cell_of(p, nc);
    atom_cell[i] = c;
    slot[i] = atomicAdd(&count[c], 1);
}

// Exclusive scan of count[0..n) into start[0..n] by one CTA of 1024 threads,
// in tiles of 8 consecutive values per thread (two 16-byte loads and stores);
// start[n] is the total. With flags: overflow if the total exceeds cap, and
// flags[flag_max] = max(total).
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;

__global__ void __launch_bounds__(kScanThreads) k_scan_1cta(int n, const int* __restrict__ count,
                                                            int* __restrict__ start, long long cap,
                                                            int* __restrict__ flags, int flag_max, const int* gate) {
    if (gated_off(gate)) return;
    __shared__ int warp_sums[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    constexpr int nw = kScanThreads / 32;
    int carry = 0;
    for (int base = 0; base < n; base += kScanThreads * kScanPer) {
        const int i0 = base + t * kScanPer;
        int v[kScanPer];
        if (i0 + kScanPer <= n) {
            const int4 a = *reinterpret_cast<const int4*>(count + i0);
            const int4 b = *reinterpret_cast<const int4*>(count + i0 + 4);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < kScanPer; ++k) v[k] = i0 + k < n ? count[i0 + k] : 0;
        }
        int local = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) local += v[k];
        int incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[w] = incl;
        __syncthreads();
        if (w == 0) {
            int sum = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, sum, o);
                if (lane >= o) sum += y;
            }
            warp_sums[lane] = sum;
        }
        __syncthreads();
        int e = carry + incl - local + (w > 0 ? warp_sums[w - 1] : 0);
        int o[kScanPer];
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) { o[k] = e; e += v[k]; }
        if (i0 + kScanPer <= n) {
            *reinterpret_cast<int4*>(start + i0) = make_int4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<int4*>(start + i0 + 4) = make_int4(o[4], o[5], o[6], o[7]);
        } else {
#pragma unroll
            for (int k = 0; k < kScanPer; ++k)
                if (i0 + k < n) start[i0 + k] = o[k];
        }
        carry += warp_sums[nw - 1];
        __syncthreads();                                   // warp_sums is rewritten by the next tile
    }
    if (t == 0) {
        start[n] = carry;
        if (flags) {
            if ((long long)carry > cap) atomicOr(&flags[kFlagOverflow], 1);
            atomicMax(&flags[flag_max], carry);
        }
    }
}

// Fixed-capacity cells (fresh lists): every atom into its cell.
__global__ void k_cell_place(int n, const uint4* __restrict__ q, CellPlace cp, int* __restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    place_in_cell(cp, i, q[i], flags);
}

// Atoms in cell order, with their fixed-point positions beside them (the
// builder then reads each cell's candidates contiguously; the fourth word
// holds the atom index instead of the system) and each atom's own place in
// that order.
__global__ void k_cell_fill(int n, const int* __restrict__ atom_cell, const int* __restrict__ slot,
                            const int* __restrict__ start, int* __restrict__ cell_atoms, const uint4* __restrict__ q,
                            uint4* __restrict__ cell_q, int* __restrict__ atom_pos, const int* gate) {
    if (gated_off(gate)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int pos = start[atom_cell[i]] + slot[i];
    const uint4 qi = q[i];
    cell_atoms[pos] = i;
    cell_q[pos] = make_uint4(qi.x, qi.y, qi.z, (unsigned int)i);
    atom_pos[i] = pos;
}

void launch_cells_gated(int n_atoms, const uint4* q, int nc, int* cell_count, int* cell_start,
                        int* cell_atoms, int* atom_cell, int* atom_slot, uint4* cell_q, int* atom_pos,
                        const int* gate, cudaStream_t s) {
    int n_cells = nc * nc * nc;
    if (n_atoms == 0) return;
    k_cell_clear<<<std::min(152, (n_cells + 255) / 256), 256, 0, s>>>(n_cells, cell_count, gate);
    int g = (n_atoms + 255) / 256;
    k_cell_count<<<g, 256, 0, s>>>(n_atoms, q, nc, cell_count, atom_cell, atom_slot, gate);
    k_scan_1cta<<<1, kScanThreads, 0, s>>>(n_cells, cell_count, cell_start, 0, nullptr, 0, gate);
    k_cell_fill<<<g, 256, 0, s>>>(n_atoms, atom_cell, atom_slot, cell_start, cell_atoms, q, cell_q, atom_pos, gate);
    count_launch(4);
}


// ------------------------------------------------------------ neighbours
// Exact FP64 decision, operation by operation (no contraction).
__device__ __forceinline__ bool exact_inside(const double* __restrict__ x, int n, int i, int j,
                                             double L, double rc) {
    double d[3];
    for (int c = 0; c < 3; ++c) {
        double dx = __dsub_rn(x[(size_t)c * n + j], x[(size_t)c * n + i]);
        if (L > 0.0) {
            double k = rint(__ddiv_rn(dx, L));
            dx = __dsub_rn(dx, __dmul_rn(L, k));
        }
        d[c] = dx;
    }
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
    return d2 < __dmul_rn(rc, rc);
}

constexpr int kNbrWarps = 8;
constexpr int kChunkBlocks = 32;      // build blocks per chunk of the folded row scan
// dynamic shared memory the builder may use: the per-block maximum (227 KB)
// less room for its static arrays
constexpr int kNbrDynSmemMax = 226 * 1024;

// One warp per atom i: enumerate candidates (27 cells, or every atom of the
// system), keep those inside the cutoff, sort the row by j (rank sort) and
// store it in the fixed-capacity staging array.
__device__ __forceinline__ void nbr_build_row(const NbrArgs& a, int* smem_i, int& n_out);

// With block_sum set, the block also publishes its pair count (the sum of its
// kNbrWarps rows) for the compaction's folded scan.
__global__ void __launch_bounds__(kNbrWarps * 32) k_nbr_build(NbrArgs a) {
    if (gated_off(a.gate)) return;
    extern __shared__ int smem_i[];
    __shared__ int rows_n[kNbrWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int n_out = 0;
    if (blockIdx.x * kNbrWarps + w < a.n_atoms) nbr_build_row(a, smem_i, n_out);
    if (!a.block_sum) return;
    if (lane == 0) rows_n[w] = n_out;
    __syncthreads();
    if (threadIdx.x == 0) {
        int sum = 0;
        for (int k = 0; k < kNbrWarps; ++k) sum += rows_n[k];
        a.block_sum[blockIdx.x] = sum;
        atomicAdd(&a.chunk_sum[blockIdx.x / kChunkBlocks], sum);    // integer: exact in any order
    }
}

// Row of atom i = blockIdx.x * kNbrWarps + warp; n_out receives its length.
__device__ __forceinline__ void nbr_build_row(const NbrArgs& a, int* smem_i, int& n_out) {
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* row = smem_i + w * (a.row_cap + 64);
    int* cstart = row + a.row_cap;       // 27 cell starts
    int* cpre = cstart + 28;             // 28 prefix sums
    int i = blockIdx.x * kNbrWarps + w;
    uint4 qi = a.q[i];
    int s = (int)qi.w;
    float qscale = a.frame[s].qscale;
    double L = a.box[s];
    if (a.xref && lane < 3) a.xref[(size_t)lane * a.n_atoms + i] = a.x[(size_t)lane * a.n_atoms + i];
    int total;
    int base = 0;
    if (a.nc > 0) {
        int nc = a.nc;
        int cx = cell_coord(qi.x, nc), cy = cell_coord(qi.y, nc), cz = cell_coord(qi.z, nc);
        int cnt = 0, st = 0;
        if (lane < 27) {
            int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
            // periodic neighbour cells (the offsets are -1, 0 or 1: one wrap at most)
            auto wrap = [nc](int t) { return t < 0 ? t + nc : (t >= nc ? t - nc : t); };
            int x2 = wrap(cx + dx), y2 = wrap(cy + dy), z2 = wrap(cz + dz);
            int c = ((s * nc + z2) * nc + y2) * nc + x2;       // the system's own cells
            c = DMTS_IDX(c, a.ccap > 0 ? (long long)a.n_cells : (long long)nc * nc * nc * a.n_sys, a.flags);
            if (a.ccap > 0) {                        // fixed-capacity cells
                st = c * a.ccap;
                cnt = min(a.cell_count[c], a.ccap);
            } else {
                st = a.cell_start[c];
                cnt = a.cell_start[c + 1] - st;
            }
            // A neighbour cell whose box lies entirely beyond the cutoff has no
            // pair: its distance from atom i is at least that of the faces of
            // i's own cell it lies behind (fixed-point units, then A). The cells
            // are wider than the cutoff, so a farther periodic image of the cell
            // is out of range too; the 0.1 % margin covers the FP32 rounding of
            // the bound. About a third of the candidates of a 27-cell scan are
            // skipped when the cells are barely wider than the cutoff.
            const float W = 4294967296.0f / (float)nc;
            auto face = [W](int d, int cc, unsigned int q) {
                return d == 0 ? 0.f : (d < 0 ? (float)q - (float)cc * W : (float)(cc + 1) * W - (float)q);
            };
            const float fx = face(dx, cx, qi.x), fy = face(dy, cy, qi.y), fz = face(dz, cz, qi.z);
            if ((fx * fx + fy * fy + fz * fz) * (qscale * qscale) > a.rc2_hi * 1.001f) cnt = 0;
        }
        int v = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < 27) { cstart[lane] = st; cpre[lane] = v - cnt; }
        total = __shfl_sync(0xffffffffu, v, 26);
        if (lane == 0) cpre[27] = total;
        __syncwarp();
    } else {
        base = a.atom_offset[s];
        total = a.atom_offset[s + 1] - base;
    }
    int n_row = 0;
    const float rc2_lo = a.rc2_lo, rc2_hi = a.rc2_hi;
    const int my_pos = a.nc > 0 ? a.atom_pos[i] : -1;
    for (int v0 = 0; v0 < total; v0 += 32) {
        int v = v0 + lane;
        bool keep = false;
        int j = -1;
        if (v < total) {
            if (a.nc > 0) {
                int c = 0;                                   // last of the 27 cells with cpre[c] <= v
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (c + step < 27 && cpre[c + step] <= v) c += step;
                // candidates in cell order: consecutive lanes read consecutive positions
                const int pos = DMTS_IDX(cstart[c] + (v - cpre[c]),
                                         a.ccap > 0 ? (long long)a.n_cells * a.ccap : (long long)a.n_atoms, a.flags);
                if (pos != my_pos) {
                    const uint4 qc = a.cell_q[pos];          // position and atom index in one load
                    float3 r = edge_vec(qi, qc, qscale);
                    float d2 = r.x * r.x + r.y * r.y + r.z * r.z;
                    if (d2 < rc2_lo) {
                        keep = true;
                        j = DMTS_IDX((int)qc.w, a.n_atoms, a.flags);
                    } else if (d2 <= rc2_hi) {
                        j = DMTS_IDX((int)qc.w, a.n_atoms, a.flags);
                        keep = a.exact ? exact_inside(a.x, a.n_atoms, i, j, L, a.rc) : true;
                    }
                }
            } else {
                j = base + v;
                if (j != i) {
                    float3 r = edge_vec(qi, a.q[j], qscale);
                    float d2 = r.x * r.x + r.y * r.y + r.z * r.z;
                    if (d2 < rc2_lo) keep = true;
                    else if (d2 <= rc2_hi) keep = a.exact ? exact_inside(a.x, a.n_atoms, i, j, L, a.rc) : true;
                }
            }
        }
        unsigned int m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = n_row + __popc(m & ((1u << lane) - 1u));
            if (pos < a.row_cap) row[pos] = j;
        }
        n_row += __popc(m);
    }
    __syncwarp();
    if (lane == 0) {
        if (n_row > a.row_cap) {                     // the capacity grows from the longest overflowing row
            atomicMax(&a.flags[a.flag_row], n_row);
            atomicOr(&a.flags[kFlagOverflow], 1);
        }
    }
    int n_keep = min(n_row, a.row_cap);
    int* dst = a.nbr_tmp + (size_t)i * a.row_cap;
    if (n_keep > 32 && n_keep <= 64) {
        // 33 to 64 kept pairs: a bitonic sort of 64 keys, two per lane (key
        // e = lane + 32 h in register h), padded with INT_MAX; the rank sort
        // below would take n_keep shared-memory reads per key
        int v[2];
        v[0] = row[lane];
        v[1] = lane + 32 < n_keep ? row[lane + 32] : 0x7fffffff;
        for (int k = 2; k <= 64; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                if (jj == 32) {                              // partner: the other register of this lane
                    const int lo = min(v[0], v[1]), hi = max(v[0], v[1]);
                    v[0] = lo;                                // k = 64: ascending over the whole row
                    v[1] = hi;
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int e = lane + 32 * h;
                        const int o = __shfl_xor_sync(0xffffffffu, v[h], jj);
                        const bool up = (e & k) == 0;         // this k-block sorts ascending
                        const bool low = (e & jj) == 0;       // this key is the lower of its pair
                        v[h] = (low == up) ? min(v[h], o) : max(v[h], o);
                    }
                }
            }
        }
        dst[lane] = v[0];
        if (lane + 32 < n_keep) dst[lane + 32] = v[1];
    } else {
        for (int k = lane; k < n_keep; k += 32) {
            int jk = row[k];
            int rank = 0;
            for (int m2 = 0; m2 < n_keep; ++m2) rank += (row[m2] < jk);
            dst[rank] = jk;
        }
    }
    if (lane == 0) a.nbr_cnt[i] = n_keep;
    n_out = n_keep;
}

// Compaction with the row scan folded in (fresh lists, block_sum set): block
// b holds the kCompactAtoms atoms of build blocks kCompactBlocks b ..
// + kCompactBlocks - 1 (one chunk of the scan holds whole compaction
// blocks). Warp 0 adds the pair counts of every earlier chunk of
// kChunkBlocks build blocks and of the earlier build blocks of this chunk,
// then scans the block's own rows; each warp copies four consecutive rows
// as one range of pairs (the rows follow each other in the pair list).
// row_ptr[n] and the capacity checks come from the warp of the last atom.
// The last block to finish clears the chunk sums and the ticket for the
// next build.
constexpr int kCompactAtoms = 32;
constexpr int kCompactBlocks = kCompactAtoms / kNbrWarps;
constexpr int kCompactRows = kCompactAtoms / kNbrWarps;   // rows per warp
static_assert(kCompactAtoms == 32, "warp 0 scans one row per lane");
static_assert(kChunkBlocks % kCompactBlocks == 0, "a compaction block lies in one chunk");

__global__ void __launch_bounds__(kNbrWarps * 32) k_nbr_compact_scan(NbrArgs a) {
    __shared__ int row_beg[kCompactAtoms + 1];
    if (a.ccap > 0)
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_cells; k += gridDim.x * blockDim.x)
            a.cell_count[k] = 0;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b0 = blockIdx.x * kCompactBlocks, chunk = b0 / kChunkBlocks;
    const int atom0 = blockIdx.x * kCompactAtoms;
    if (w == 0) {
        long long sum = 0;
        for (int c = lane; c < chunk; c += 32) sum += a.chunk_sum[c];
        for (int c = chunk * kChunkBlocks + lane; c < b0; c += 32) sum += a.block_sum[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const int cnt = atom0 + lane < a.n_atoms ? a.nbr_cnt[atom0 + lane] : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        row_beg[lane] = (int)sum + incl - cnt;
        if (lane == 31) row_beg[32] = (int)sum + incl;
    }
    __syncthreads();
    const int r0 = kCompactRows * w, i0 = atom0 + r0;
    if (i0 < a.n_atoms) {
        const int nr = min(kCompactRows, a.n_atoms - i0);
        const int beg = row_beg[r0], end = row_beg[r0 + nr];
        if (lane < nr) a.row_ptr[i0 + lane] = row_beg[r0 + lane];
        if (i0 + nr == a.n_atoms && lane == 0) {
            a.row_ptr[a.n_atoms] = end;
            if ((long long)end > a.e_cap) atomicOr(&a.flags[kFlagOverflow], 1);
            atomicMax(&a.flags[kFlagMaxE0 + a.which], end);
        }
        for (int e = beg + lane; e < end; e += 32) {
            int r = 0;                                   // the last of the warp's rows starting at or before e
#pragma unroll
            for (int q = 1; q < kCompactRows; ++q)
                if (q < nr && row_beg[r0 + q] <= e) r = q;
            if ((long long)e < a.e_cap) {
                const int i = i0 + r;
                a.col[e] = a.nbr_tmp[(size_t)i * a.row_cap + (e - row_beg[r0 + r])];
                a.recv[e] = i;
            }
        }
    }
    // every block has read the chunk sums: the last one clears them
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.ticket, 1u) == gridDim.x - 1) {
            const int n_build = (a.n_atoms + kNbrWarps - 1) / kNbrWarps;
            const int n_chunks = (n_build + kChunkBlocks - 1) / kChunkBlocks;
            for (int c = 0; c < n_chunks; ++c) a.chunk_sum[c] = 0;
            *a.ticket = 0u;
        }
    }
}

__global__ void k_nbr_compact(NbrArgs a) {
    // fixed-capacity cells: the counters start the next build at zero
    if (a.ccap > 0)
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_cells; k += gridDim.x * blockDim.x)
            a.cell_count[k] = 0;
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= a.n_atoms) return;
    int i = w;
    int beg = a.row_ptr[i], cnt = a.nbr_cnt[i];
    const int* src = a.nbr_tmp + (size_t)i * a.row_cap;
    for (int k = lane; k < cnt; k += 32) {
        long long e = (long long)beg + k;
        if (e < a.e_cap) {
            a.col[e] = src[k];
            a.recv[e] = i;
        }
    }
}

// One warp per atom: keep the candidates of row i (ascending j) that pass the
// test, in order, so the output row is ascending as well. a.exact selects the
// exact cutoff test of the final pair set or the plain FP32 bound used to
// derive one model's candidate rows from the other's.
__global__ void __launch_bounds__(256) k_row_filter(NbrArgs a) {
    if (gated_off(a.gate)) return;
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= a.n_atoms) return;
    const uint4 qi = a.q[i];
    const int s = (int)qi.w;
    const float qscale = a.frame[s].qscale;
    const double L = a.box[s];
    const int cnt = a.src_cnt[i];
    const int* src = a.src_rows + (size_t)i * a.src_cap;
    int* dst = a.nbr_tmp + (size_t)i * a.row_cap;
    const float rc2_lo = a.rc2_lo, rc2_hi = a.rc2_hi;
    int n_row = 0;
    for (int v0 = 0; v0 < cnt; v0 += 32) {
        const int v = v0 + lane;
        bool keep = false;
        int j = -1;
        if (v < cnt) {
            j = src[v];
            float3 r = edge_vec(qi, a.q[j], qscale);
            float d2 = r.x * r.x + r.y * r.y + r.z * r.z;
            if (d2 < rc2_lo) keep = true;
            else if (d2 <= rc2_hi) keep = a.exact ? exact_inside(a.x, a.n_atoms, i, j, L, a.rc) : true;
        }
        const unsigned int m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int pos = n_row + __popc(m & ((1u << lane) - 1u));
            if (pos < a.row_cap) dst[pos] = j;
        }
        n_row += __popc(m);
    }
    if (lane == 0) {
        if (n_row > a.row_cap) {                     // the capacity grows from the longest overflowing row
            atomicMax(&a.flags[a.flag_row], n_row);
            atomicOr(&a.flags[kFlagOverflow], 1);
        }
        a.nbr_cnt[i] = min(n_row, a.row_cap);
    }
}

// Largest squared displacement since the rebuild, reduced over CTAs; the
// last CTA to finish takes the decision (vl_block_decide).
__global__ void __launch_bounds__(256) k_vl_check(int n, const double* __restrict__ x, const int* __restrict__ sys,
                                                  const double* __restrict__ box, VerletCheck vc) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = fmax(m, vl_disp2(x, vc.xref, (size_t)n, (size_t)i, box[sys[i]], vc.thr2));
    vl_block_decide(m, vc);
}

void launch_vl_check(int n_atoms, const double* x, const int* sys_of_atom, const double* box,
                     const VerletCheck& vc, cudaStream_t s) {
    const int g = std::max(1, std::min(4 * 152, (n_atoms + 255) / 256));
    k_vl_check<<<g, 256, 0, s>>>(n_atoms, x, sys_of_atom, box, vc);
    count_launch();
}

void launch_row_filter(const NbrArgs& a, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    k_row_filter<<<(a.n_atoms * 32 + 255) / 256, 256, 0, s>>>(a);
    count_launch();
}

void launch_vl_build(const NbrArgs& a, cudaStream_t s) {
    if (a.n_atoms == 0) return;
    smem_opt_in((const void*)k_nbr_build, kNbrDynSmemMax);
    int blocks = (a.n_atoms + kNbrWarps - 1) / kNbrWarps;
    size_t smem = sizeof(int) * (size_t)kNbrWarps * (a.row_cap + 64);
    k_nbr_build<<<blocks, kNbrWarps * 32, smem, s>>>(a);
    count_launch();
}

void launch_vl_filter(const NbrArgs& a, cudaStream_t s) {
    if (a.n_atoms == 0) {
        cudaMemsetAsync(a.row_ptr, 0, sizeof(int), s);
        return;
    }
    k_row_filter<<<(a.n_atoms * 32 + 255) / 256, 256, 0, s>>>(a);
    k_scan_1cta<<<1, kScanThreads, 0, s>>>(a.n_atoms, a.nbr_cnt, a.row_ptr, a.e_cap, a.flags,
                                          kFlagMaxE0 + a.which, nullptr);
    k_nbr_compact<<<(a.n_atoms * 32 + 255) / 256, 256, 0, s>>>(a);
    count_launch(3);
}

void launch_neighbors(const NbrArgs& a, cudaStream_t s) {
    if (a.n_atoms == 0) {
        cudaMemsetAsync(a.row_ptr, 0, sizeof(int), s);
        return;
    }
    if (a.nc > 0 && a.ccap > 0 && !a.placed) {
        const CellPlace cp{a.nc, a.ccap, a.cell_count, const_cast<int*>(a.cell_atoms),
                           const_cast<uint4*>(a.cell_q), const_cast<int*>(a.atom_pos), kFlagMaxCell0 + a.which};
        k_cell_place<<<(a.n_atoms + 255) / 256, 256, 0, s>>>(a.n_atoms, a.q, cp, a.flags);
        count_launch();
    }
    smem_opt_in((const void*)k_nbr_build, kNbrDynSmemMax);
    int blocks = (a.n_atoms + kNbrWarps - 1) / kNbrWarps;
    size_t smem = sizeof(int) * (size_t)kNbrWarps * (a.row_cap + 64);
    k_nbr_build<<<blocks, kNbrWarps * 32, smem, s>>>(a);
    if (a.block_sum) {                     // row scan folded into the compaction
        k_nbr_compact_scan<<<(a.n_atoms + kCompactAtoms - 1) / kCompactAtoms, kNbrWarps * 32, 0, s>>>(a);
        count_launch(2);
        return;
    }
    k_scan_1cta<<<1, kScanThreads, 0, s>>>(a.n_atoms, a.nbr_cnt, a.row_ptr, a.e_cap, a.flags,
                                          kFlagMaxE0 + a.which, nullptr);
    k_nbr_compact<<<(a.n_atoms * 32 + 255) / 256, 256, 0, s>>>(a);
    count_launch(3);
}

}  // namespace dmts
