// dmts_neighbors_noalloc: the neighbour list of one system without any
// device allocation.
//
// Some callers cannot call cudaMalloc: an MD engine that owns every byte of
// device memory through its own pool and hands plug-ins pre-allocated
// buffers, or code running under a fixed memory budget where an allocation
// would synchronise the device or fail. For them this entry point keeps its
// scratch (fixed-point
// positions, cell list, per-atom counts) in one file-scope static device
// array of fixed size, reserved once per device when the library is loaded
// and held until the process exits. The caller passes device buffers for the
// positions and for the CSR output.
//
// The array's name is a host-side stand-in in host code, not a device
// address, so the host resolves its device address with cudaGetSymbolAddress,
// once per device, on the first call made with that device current.
//
// Result: the same pair set and row order as dmts_neighbors (two passes, count
// then fill, instead of a staging array).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "../../include/dmts.h"
#include "internal.cuh"

namespace {

constexpr int kMaxAtoms = DMTS_NOALLOC_MAX_ATOMS;
constexpr int kMaxCellsPerDim = 32;
constexpr int kMaxCells = kMaxCellsPerDim * kMaxCellsPerDim * kMaxCellsPerDim;
constexpr int kRowMax = 256;          // longest row the fill pass sorts in shared memory
constexpr int kWarps = 8;

// Carving of the scratch array (byte offsets, 256-aligned).
constexpr size_t align256(size_t n) { return (n + 255) / 256 * 256; }
constexpr size_t kOffQ = 0;                                                    // uint4 [kMaxAtoms]
constexpr size_t kOffCell = kOffQ + align256(sizeof(uint4) * kMaxAtoms);       // int [kMaxAtoms]
constexpr size_t kOffSlot = kOffCell + align256(sizeof(int) * kMaxAtoms);      // int [kMaxAtoms]
constexpr size_t kOffCellAtoms = kOffSlot + align256(sizeof(int) * kMaxAtoms); // int [kMaxAtoms]
constexpr size_t kOffCnt = kOffCellAtoms + align256(sizeof(int) * kMaxAtoms);  // int [kMaxAtoms]
constexpr size_t kOffCellCount = kOffCnt + align256(sizeof(int) * kMaxAtoms);  // int [kMaxCells]
constexpr size_t kOffCellStart = kOffCellCount + align256(sizeof(int) * kMaxCells);  // int [kMaxCells + 1]
constexpr size_t kOffFrame = kOffCellStart + align256(sizeof(int) * (kMaxCells + 1));  // Frame
constexpr size_t kOffFlags = kOffFrame + align256(sizeof(dmts::Frame));        // int [4]
constexpr size_t kScratchBytes = kOffFlags + 256;

// The scratch: one static device array (about 0.8 MB), shared by every call.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

int na_fail(int code, const char* fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    dmts::set_error_message(buf);
    return code;
}

struct Scratch {
    uint4* q;
    int *cell, *slot, *cell_atoms, *cnt, *cell_count, *cell_start, *flags;
    dmts::Frame* frame;
};

Scratch carve(unsigned char* base) {
    Scratch s;
    s.q = reinterpret_cast<uint4*>(base + kOffQ);
    s.cell = reinterpret_cast<int*>(base + kOffCell);
    s.slot = reinterpret_cast<int*>(base + kOffSlot);
    s.cell_atoms = reinterpret_cast<int*>(base + kOffCellAtoms);
    s.cnt = reinterpret_cast<int*>(base + kOffCnt);
    s.cell_count = reinterpret_cast<int*>(base + kOffCellCount);
    s.cell_start = reinterpret_cast<int*>(base + kOffCellStart);
    s.frame = reinterpret_cast<dmts::Frame*>(base + kOffFrame);
    s.flags = reinterpret_cast<int*>(base + kOffFlags);
    return s;
}

// Per-device address of g_scratch, resolved once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

int scratch_base(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return na_fail(DMTS_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(DMTS_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_base[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_base[dev];
    return DMTS_OK;
}

// ------------------------------------------------------------ kernels
__device__ __forceinline__ int cell_of(unsigned int qc, int nc) {
    return (int)(((unsigned long long)qc * (unsigned long long)nc) >> 32);
}

__device__ __forceinline__ unsigned int fixed(double v, double o, double inv) {
    long long k = (long long)floor((v - o) * inv);
    return (unsigned int)(k & 0xffffffffll);
}

// Non-periodic frame: origin = lower corner, Q = power of two >= 2 (extent + 2 rc + 1).
__global__ void k_frame_open(int n, const double* __restrict__ x, double rc, dmts::Frame* frame) {
    __shared__ double lo_s[3][32], hi_s[3][32];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], x[3 * (size_t)i + c]);
            hi[c] = fmax(hi[c], x[3 * (size_t)i + c]);
        }
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; ++c) { lo_s[c][w] = lo[c]; hi_s[c][w] = hi[c]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ext = 0.0, o3[3];
        for (int c = 0; c < 3; ++c) {
            double a = 1e300, b = -1e300;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a = fmin(a, lo_s[c][k]); b = fmax(b, hi_s[c][k]); }
            o3[c] = a;
            ext = fmax(ext, b - a);
        }
        double need = 2.0 * (ext + 2.0 * rc + 1.0), Q = 1.0;
        while (Q < need) Q *= 2.0;
        dmts::Frame f;
        f.ox = o3[0]; f.oy = o3[1]; f.oz = o3[2];
        f.inv = 4294967296.0 / Q;
        f.qscale = (float)(Q / 4294967296.0);
        f.pad = 0.f;
        *frame = f;
    }
}

__global__ void k_quant(int n, const double* __restrict__ x, const dmts::Frame* __restrict__ frame,
                        uint4* __restrict__ q) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dmts::Frame f = *frame;
    q[i] = make_uint4(fixed(x[3 * (size_t)i], f.ox, f.inv), fixed(x[3 * (size_t)i + 1], f.oy, f.inv),
                      fixed(x[3 * (size_t)i + 2], f.oz, f.inv), 0u);
}

__global__ void k_cells(int n, const uint4* __restrict__ q, int nc, int* __restrict__ count,
                        int* __restrict__ cell, int* __restrict__ slot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 p = q[i];
    int c = (cell_of(p.z, nc) * nc + cell_of(p.y, nc)) * nc + cell_of(p.x, nc);
    cell[i] = c;
    slot[i] = atomicAdd(&count[c], 1);
}

// exclusive scan of count[0..n) into start[0..n], one CTA of 1024 threads
__global__ void k_scan(int n, const int* __restrict__ count, int* __restrict__ start) {
    __shared__ int ws[32];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int per = (n + blockDim.x - 1) / blockDim.x;
    int b = t * per, e = min(n, b + per);
    int local = 0;
    for (int k = b; k < e; ++k) local += count[k];
    int v = local;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    int run = v - local + (w > 0 ? ws[w - 1] : 0);
    for (int k = b; k < e; ++k) {
        start[k] = run;
        run += count[k];
    }
    if (t == blockDim.x - 1) start[n] = run;
}

__global__ void k_fill_cells(int n, const int* __restrict__ cell, const int* __restrict__ slot,
                             const int* __restrict__ start, int* __restrict__ cell_atoms) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cell_atoms[start[cell[i]] + slot[i]] = i;
}

struct PassArgs {
    int n;
    const double* x;        // caller's AoS positions [n][3]
    double L;               // > 0 periodic
    double rc;
    float rc2_lo, rc2_hi;
    int nc;                 // 0: all pairs
    Scratch s;
    const int* row_ptr;     // fill pass: caller's output from the count pass
    int* col;
    long long capacity;
};

__device__ __forceinline__ bool inside_fp64(const double* __restrict__ x, int i, int j, double L, double rc) {
    double d[3];
    for (int c = 0; c < 3; ++c) {
        double dx = __dsub_rn(x[3 * (size_t)j + c], x[3 * (size_t)i + c]);
        if (L > 0.0) dx = __dsub_rn(dx, __dmul_rn(L, rint(__ddiv_rn(dx, L))));
        d[c] = dx;
    }
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
    return d2 < __dmul_rn(rc, rc);
}

// Warp per atom. fill == false: count the row; fill == true: gather, rank-sort
// and write the row at row_ptr[i].
template <bool Fill>
__global__ void __launch_bounds__(kWarps * 32) k_pass(PassArgs a) {
    __shared__ int rows[kWarps][kRowMax];
    __shared__ int cst[kWarps][28], cpre[kWarps][28];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i = blockIdx.x * kWarps + w;
    if (i >= a.n) return;
    uint4 qi = a.s.q[i];
    float qs = a.s.frame->qscale;
    int total;
    if (a.nc > 0) {
        int nc = a.nc;
        int cx = cell_of(qi.x, nc), cy = cell_of(qi.y, nc), cz = cell_of(qi.z, nc);
        int cnt = 0, st = 0;
        if (lane < 27) {
            int x2 = (cx + lane % 3 - 1 + nc) % nc, y2 = (cy + (lane / 3) % 3 - 1 + nc) % nc,
                z2 = (cz + lane / 9 - 1 + nc) % nc;
            int c = (z2 * nc + y2) * nc + x2;
            st = a.s.cell_start[c];
            cnt = a.s.cell_start[c + 1] - st;
        }
        int v = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < 27) { cst[w][lane] = st; cpre[w][lane] = v - cnt; }
        total = __shfl_sync(0xffffffffu, v, 26);
        if (lane == 0) cpre[w][27] = total;
        __syncwarp();
    } else {
        total = a.n;
    }
    int n_row = 0;
    for (int v0 = 0; v0 < total; v0 += 32) {
        int v = v0 + lane, j = -1;
        bool keep = false;
        if (v < total) {
            if (a.nc > 0) {
                int c = 0;
                while (c < 26 && cpre[w][c + 1] <= v) ++c;
                j = a.s.cell_atoms[cst[w][c] + (v - cpre[w][c])];
            } else {
                j = v;
            }
            if (j != i) {
                uint4 qj = a.s.q[j];
                float dx = (float)(int)(qj.x - qi.x) * qs, dy = (float)(int)(qj.y - qi.y) * qs,
                      dz = (float)(int)(qj.z - qi.z) * qs;
                float d2 = dx * dx + dy * dy + dz * dz;
                keep = d2 < a.rc2_lo || (d2 <= a.rc2_hi && inside_fp64(a.x, i, j, a.L, a.rc));
            }
        }
        unsigned int m = __ballot_sync(0xffffffffu, keep);
        if (Fill && keep) {
            int pos = n_row + __popc(m & ((1u << lane) - 1u));
            if (pos < kRowMax) rows[w][pos] = j;
        }
        n_row += __popc(m);
    }
    if (!Fill) {
        if (lane == 0) {
            a.s.cnt[i] = n_row;
            if (n_row > kRowMax) atomicOr(&a.s.flags[0], 1);
        }
        return;
    }
    __syncwarp();
    if (n_row > kRowMax) return;   // reported by the count pass
    long long beg = a.row_ptr[i];
    for (int k = lane; k < n_row; k += 32) {
        int jk = rows[w][k], rank = 0;
        for (int m2 = 0; m2 < n_row; ++m2) rank += (rows[w][m2] < jk);
        long long e = beg + rank;
        if (e < a.capacity) a.col[e] = jk;
    }
}

}  // namespace

extern "C" DMTS_API int dmts_neighbors_noalloc(const double* x, int n_atoms, double box, double cutoff,
                                               int* row_ptr, int* col, long long capacity,
                                               long long* n_pairs, void* stream) {
    dmts::set_error_message("");
    if (!x || !row_ptr || !n_pairs || (capacity > 0 && !col))
        return na_fail(DMTS_ERR_ARG, "NULL argument");
    if (n_atoms < 0 || n_atoms > kMaxAtoms)
        return na_fail(DMTS_ERR_ARG, "n_atoms %d outside [0, %d], the size of the static scratch", n_atoms, kMaxAtoms);
    if (!(cutoff > 0) || !isfinite(cutoff) || !isfinite(box))
        return na_fail(DMTS_ERR_ARG, "cutoff must be > 0 and box finite");
    if (box > 0 && box < 2.0 * cutoff) return na_fail(DMTS_ERR_ARG, "box edge below twice the cutoff");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(DMTS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned char* base = nullptr;
    int rc = scratch_base(dev, &base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    *n_pairs = 0;
    if (n_atoms == 0) {
        e = cudaMemsetAsync(row_ptr, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? DMTS_OK : na_fail(DMTS_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    Scratch sc = carve(base);
    // the scratch keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(sc.flags, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return na_fail(DMTS_ERR_CUDA, "%s", cudaGetErrorString(e));
    int nc = 0;
    if (box > 0) {
        dmts::Frame f;
        f.ox = f.oy = f.oz = 0.0;
        f.inv = 4294967296.0 / box;
        f.qscale = (float)(box / 4294967296.0);
        f.pad = 0.f;
        e = cudaMemcpyAsync(sc.frame, &f, sizeof f, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // f lives on this stack frame
        if (e != cudaSuccess) return na_fail(DMTS_ERR_CUDA, "%s", cudaGetErrorString(e));
        nc = (int)floor(box / (cutoff * (1.0 + 1e-9) + 1e-6));
        if (nc > kMaxCellsPerDim) nc = kMaxCellsPerDim;   // larger cells stay correct
        if (nc < 3) nc = 0;
    } else {
        k_frame_open<<<1, 1024, 0, s>>>(n_atoms, x, cutoff, sc.frame);
    }
    int g = (n_atoms + 255) / 256;
    k_quant<<<g, 256, 0, s>>>(n_atoms, x, sc.frame, sc.q);
    if (nc > 0) {
        int ncell = nc * nc * nc;
        e = cudaMemsetAsync(sc.cell_count, 0, sizeof(int) * ncell, s);
        if (e != cudaSuccess) return na_fail(DMTS_ERR_CUDA, "%s", cudaGetErrorString(e));
        k_cells<<<g, 256, 0, s>>>(n_atoms, sc.q, nc, sc.cell_count, sc.cell, sc.slot);
        k_scan<<<1, 1024, 0, s>>>(ncell, sc.cell_count, sc.cell_start);
        k_fill_cells<<<g, 256, 0, s>>>(n_atoms, sc.cell, sc.slot, sc.cell_start, sc.cell_atoms);
    }
    PassArgs pa;
    pa.n = n_atoms;
    pa.x = x;
    pa.L = box > 0 ? box : 0.0;
    pa.rc = cutoff;
    pa.rc2_lo = (float)(cutoff * cutoff * (1.0 - 1e-5));
    pa.rc2_hi = (float)(cutoff * cutoff * (1.0 + 1e-5));
    pa.nc = nc;
    pa.s = sc;
    pa.row_ptr = row_ptr;
    pa.col = col;
    pa.capacity = capacity;
    int blocks = (n_atoms + kWarps - 1) / kWarps;
    k_pass<false><<<blocks, kWarps * 32, 0, s>>>(pa);
    k_scan<<<1, 1024, 0, s>>>(n_atoms, sc.cnt, row_ptr);
    k_pass<true><<<blocks, kWarps * 32, 0, s>>>(pa);
    int total = 0, flag = 0;
    e = cudaMemcpyAsync(&total, row_ptr + n_atoms, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, sc.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(DMTS_ERR_CUDA, "%s", cudaGetErrorString(e));
    *n_pairs = total;
    if (flag) return na_fail(DMTS_ERR_CAPACITY, "a row has more than %d neighbours", kRowMax);
    if (total > capacity) return na_fail(DMTS_ERR_CAPACITY, "%d pairs exceed capacity %lld", total, capacity);
    return DMTS_OK;
}
