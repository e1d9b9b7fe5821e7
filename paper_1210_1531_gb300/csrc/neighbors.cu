// a1: periodic cell lists, neighbour lists (the BSR pattern) and cluster lists.
//
// The pattern of H and S is every atom pair within r_cut (self included); the cluster of atom J
// is every atom within r_cluster. Both follow from the locality that makes the method order-N
// (each column touches only the cluster around its atom) and from the local, redundant build
// of H and S (data-communication saving, item I of the computational issues). Rows come out
// sorted ascending; the distance test uses single IEEE operations in a fixed order so that the
// lists are reproducible bit for bit.
#include "internal.h"

namespace elses {

// ------------------------------------------------------------------ exclusive scan (int)
// out[0..n] with out[0] = 0 and out[n] = total; one CTA, chunked; deterministic.
__global__ void k_scan_exclusive(const int* __restrict__ in, int* __restrict__ out, int n) {
    __shared__ long long part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int b = min(n, t * chunk), e = min(n, b + chunk);
    long long s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        long long v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (int i = b; i < e; ++i) {
        out[i] = (int)run;
        run += in[i];
    }
    if (t == T - 1) out[n] = (int)part[T - 1];
}

void scan_exclusive(const int* in, int* out, int n, cudaStream_t st) {
    k_scan_exclusive<<<1, 1024, 0, st>>>(in, out, n);
}

__global__ void k_check_finite(const double* __restrict__ x, int count, int* __restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && !isfinite(x[i])) flag(status, DEV_NONFINITE);
}

void check_finite(const double* x, int count, int* status, cudaStream_t st) {
    k_check_finite<<<(count + 255) / 256, 256, 0, st>>>(x, count, status);
}

// FP64 FMA throughput probe: 8 independent chains per thread, every SM busy.
__global__ void k_fp64_probe(double* out, int iters) {
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = 1.0 + 1e-3 * (threadIdx.x + q);
    const double a = 0.9999999, b = 1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += x[q];
    if (s == 12345.678) out[blockIdx.x] = s;   // keeps the chains live
}

int probe_fp64(double* gflops, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * 64 * sms);
    if (e != cudaSuccess) return (int)e;
    const int blocks = 8 * sms, threads = 256, iters = 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_fp64_probe<<<blocks, threads, 0, st>>>(out, 64);   // warm-up
    cudaEventRecord(a, st);
    k_fp64_probe<<<blocks, threads, 0, st>>>(out, iters);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e9;
    return 0;
}

// ------------------------------------------------------------------ cell grid
__device__ __forceinline__ int cell_coord(double x, double L, double len, int nc) {
    double xw = x - L * floor(x / L);
    int c = (int)floor(xw / len);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_count(const double* __restrict__ pos, int n, CellGrid g,
                             int* __restrict__ cell_of, int* __restrict__ cell_count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = cell_coord(pos[3 * i + 0], g.L[0], g.len[0], g.nc[0]);
    int cy = cell_coord(pos[3 * i + 1], g.L[1], g.len[1], g.nc[1]);
    int cz = cell_coord(pos[3 * i + 2], g.L[2], g.len[2], g.nc[2]);
    int c = (cx * g.nc[1] + cy) * g.nc[2] + cz;
    cell_of[i] = c;
    atomicAdd(&cell_count[c], 1);
}

__global__ void k_cell_fill(int n, const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                            int* __restrict__ cursor, int* __restrict__ cell_atoms) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_of[i];
    int slot = atomicAdd(&cursor[c], 1);
    cell_atoms[cell_start[c] + slot] = i;
}

// Sort the atoms of each cell ascending (insertion sort; cells hold tens of atoms).
__global__ void k_cell_sort(int ncell, const int* __restrict__ cell_start, int* __restrict__ cell_atoms) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = cell_start[c], e = cell_start[c + 1];
    for (int i = b + 1; i < e; ++i) {
        int v = cell_atoms[i];
        int k = i - 1;
        while (k >= b && cell_atoms[k] > v) {
            cell_atoms[k + 1] = cell_atoms[k];
            --k;
        }
        cell_atoms[k + 1] = v;
    }
}

// Stencil of cell offsets along one axis: all cells when the reach wraps onto itself.
__device__ __forceinline__ void axis_range(int c, int reach, int nc, int& first, int& count, bool& absolute) {
    if (2 * reach + 1 >= nc) { first = 0; count = nc; absolute = true; }
    else { first = c - reach; count = 2 * reach + 1; absolute = false; }
}

// ------------------------------------------------------------------ list build (warp per atom)
// FILL = false: counts[i] = number of atoms within r of atom i (and max into *max_count).
// FILL = true : writes the sorted list into idx[ptr[i] ..), using a per-warp shared buffer of
//               `cap` entries (overflow sets DEV_CAPACITY and skips the row).
constexpr int kListWarps = 8;   // warps (atoms) per CTA of k_lists

template <bool FILL>
__global__ void k_lists(const double* __restrict__ pos, int n, CellGrid g,
                        const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                        const int* __restrict__ cell_atoms, double r, int reach0, int reach1,
                        int reach2, int* __restrict__ counts, int* __restrict__ max_count,
                        const int* __restrict__ ptr, int* __restrict__ idx, int cap,
                        int* __restrict__ status) {
    extern __shared__ int sbuf[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int i = blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= n) return;
    int* buf = sbuf + wib * cap;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const double r2 = __dmul_rn(r, r);
    const float fxi = (float)xi, fyi = (float)yi, fzi = (float)zi;
    const float fL[3] = {(float)g.L[0], (float)g.L[1], (float)g.L[2]};
    const float fiL[3] = {1.0f / fL[0], 1.0f / fL[1], 1.0f / fL[2]};
    // the FP32 image choice can differ from the exact one only for |d| ~ L/2, which is farther
    // than r whenever L/2 - r is not tiny; otherwise every candidate takes the exact test
    const bool pre_ok = 0.5 * g.L[0] - r > 0.01 && 0.5 * g.L[1] - r > 0.01 && 0.5 * g.L[2] - r > 0.01;
    const float r2_pre = pre_ok ? ((float)r + 0.05f) * ((float)r + 0.05f) : 3.0e38f;
    const int c = cell_of[i];
    const int ci[3] = {c / (g.nc[1] * g.nc[2]), (c / g.nc[2]) % g.nc[1], c % g.nc[2]};
    const int reach[3] = {reach0, reach1, reach2};
    int first[3], count[3];
    bool absol[3];
    for (int d = 0; d < 3; ++d) axis_range(ci[d], reach[d], g.nc[d], first[d], count[d], absol[d]);
    // candidates that pass the FP32 prefilter wait in a per-warp buffer and take the exact FP64
    // test 32 at a time with every lane busy (the FP64 pipe charges a warp instruction whatever
    // its active lanes, and few candidates of each 32 pass the prefilter)
    __shared__ int cand_buf[kListWarps][64];
    int* cb = cand_buf[wib];
    int nb = 0;
    int found = 0;
    auto exact_chunk = [&](int cnt) {
        bool hit = false;
        int j = -1;
        if (lane < cnt) {
            j = cb[lane];
            const double dx = min_image(__dsub_rn(pos[3 * j], xi), g.L[0]);
            const double dy = min_image(__dsub_rn(pos[3 * j + 1], yi), g.L[1]);
            const double dz = min_image(__dsub_rn(pos[3 * j + 2], zi), g.L[2]);
            hit = dist2_exact(dx, dy, dz) <= r2;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (FILL && hit) {
            const int slot = found + __popc(m & ((1u << lane) - 1u));
            if (slot < cap) buf[slot] = j;
        }
        found += __popc(m);
    };
    for (int a = 0; a < count[0]; ++a) {
        int cx = first[0] + a;
        if (!absol[0]) cx = (cx % g.nc[0] + g.nc[0]) % g.nc[0];
        for (int b = 0; b < count[1]; ++b) {
            int cy = first[1] + b;
            if (!absol[1]) cy = (cy % g.nc[1] + g.nc[1]) % g.nc[1];
            // the stencil's cells along z are consecutive in the cell order, so their atoms form
            // one range of cell_atoms (two where the stencil wraps around the box)
            int zlo[2], zhi[2], nr = 0;
            if (absol[2]) {
                zlo[0] = 0;
                zhi[0] = g.nc[2];
                nr = 1;
            } else {
                int lo = first[2], hi = first[2] + count[2];     // [lo, hi), count < nc
                if (lo < 0) { zlo[nr] = lo + g.nc[2]; zhi[nr] = g.nc[2]; ++nr; lo = 0; }
                else if (hi > g.nc[2]) { zlo[nr] = 0; zhi[nr] = hi - g.nc[2]; ++nr; hi = g.nc[2]; }
                zlo[nr] = lo;
                zhi[nr] = hi;
                ++nr;
            }
            for (int run = 0; run < nr; ++run) {
                const int row = (cx * g.nc[1] + cy) * g.nc[2];
                const int s0 = cell_start[row + zlo[run]], s1 = cell_start[row + zhi[run]];
                for (int base = s0; base < s1; base += 32) {
                    const int q = base + lane;
                    bool pass = false;
                    int j = -1;
                    if (q < s1) {
                        j = cell_atoms[q];
                        // FP32 prefilter (error < 1e-3 A^2 for boxes of a few hundred A): only
                        // candidates near the sphere take the exact FP64 test
                        const float fx = (float)pos[3 * j] - fxi, fy = (float)pos[3 * j + 1] - fyi,
                                    fz = (float)pos[3 * j + 2] - fzi;
                        const float gx = fx - fL[0] * rintf(fx * fiL[0]);
                        const float gy = fy - fL[1] * rintf(fy * fiL[1]);
                        const float gz = fz - fL[2] * rintf(fz * fiL[2]);
                        pass = gx * gx + gy * gy + gz * gz <= r2_pre;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, pass);
                    if (pass) cb[nb + __popc(m & ((1u << lane) - 1u))] = j;
                    nb += __popc(m);
                    __syncwarp();
                    if (nb >= 32) {          // a full chunk: test it, keep the rest (< 32)
                        exact_chunk(32);
                        const int rest = nb - 32;
                        const int v = lane < rest ? cb[32 + lane] : 0;
                        __syncwarp();
                        if (lane < rest) cb[lane] = v;
                        nb = rest;
                        __syncwarp();
                    }
                }
            }
        }
    }
    if (nb > 0) exact_chunk(nb);
    if (!FILL) {
        if (lane == 0) {
            counts[i] = found;
            atomicMax(max_count, found);
        }
        return;
    }
    __syncwarp();
    if (found > cap || found != ptr[i + 1] - ptr[i]) {
        if (lane == 0) flag(status, DEV_CAPACITY);
        return;
    }
    // rank sort (atom ids are distinct)
    const int base_out = ptr[i];
    for (int q = lane; q < found; q += 32) {
        const int v = buf[q];
        int rank = 0;
        for (int m2 = 0; m2 < found; ++m2) rank += buf[m2] < v;
        idx[base_out + rank] = v;
    }
}

template __global__ void k_lists<false>(const double*, int, CellGrid, const int*, const int*, const int*,
                                        double, int, int, int, int*, int*, const int*, int*, int, int*);
template __global__ void k_lists<true>(const double*, int, CellGrid, const int*, const int*, const int*,
                                       double, int, int, int, int*, int*, const int*, int*, int, int*);

void build_cells(const double* pos, int n, const CellGrid& g, int* cell_of, int* cell_count,
                 int* cell_start, int* cursor, int* cell_atoms, cudaStream_t st) {
    cudaMemsetAsync(cell_count, 0, sizeof(int) * g.ncell, st);
    cudaMemsetAsync(cursor, 0, sizeof(int) * g.ncell, st);
    const int T = 256;
    k_cell_count<<<(n + T - 1) / T, T, 0, st>>>(pos, n, g, cell_of, cell_count);
    scan_exclusive(cell_count, cell_start, g.ncell, st);
    k_cell_fill<<<(n + T - 1) / T, T, 0, st>>>(n, cell_of, cell_start, cursor, cell_atoms);
    k_cell_sort<<<(g.ncell + T - 1) / T, T, 0, st>>>(g.ncell, cell_start, cell_atoms);
}

void count_lists(const double* pos, int n, const CellGrid& g, const int* cell_of,
                 const int* cell_start, const int* cell_atoms, double r, int* counts,
                 int* max_count, cudaStream_t st) {
    int reach[3];
    for (int d = 0; d < 3; ++d) reach[d] = (int)ceil(r / g.len[d]);
    const int W = kListWarps;
    k_lists<false><<<(n + W - 1) / W, 32 * W, 0, st>>>(pos, n, g, cell_of, cell_start, cell_atoms, r,
                                                       reach[0], reach[1], reach[2], counts, max_count,
                                                       nullptr, nullptr, 0, nullptr);
}

void fill_lists(const double* pos, int n, const CellGrid& g, const int* cell_of,
                const int* cell_start, const int* cell_atoms, double r, const int* ptr, int* idx,
                int cap, int* status, cudaStream_t st) {
    int reach[3];
    for (int d = 0; d < 3; ++d) reach[d] = (int)ceil(r / g.len[d]);
    const int W = kListWarps;
    const size_t smem = sizeof(int) * (size_t)cap * W;
    if (smem > 48 * 1024)
        smem_at_least(k_lists<true>, smem);
    k_lists<true><<<(n + W - 1) / W, 32 * W, smem, st>>>(pos, n, g, cell_of, cell_start, cell_atoms, r,
                                                         reach[0], reach[1], reach[2], nullptr, nullptr,
                                                         ptr, idx, cap, status);
}

// Counts the pattern pairs (I, J), I in row J's list, whose atom I lies outside the cluster of J
// (clusters as sorted lists cl_idx[cl_ptr[J] ..]); the pattern is already known to be well formed.
__global__ void k_pattern_outside(int n, const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                                  const int* __restrict__ cl_ptr, const int* __restrict__ cl_idx,
                                  int* __restrict__ count) {
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= n) return;
    const int a = cl_ptr[J], b = cl_ptr[J + 1];
    int missing = 0;
    for (int e = row_ptr[J]; e < row_ptr[J + 1]; ++e) {
        const int I = col_idx[e];
        int lo = a, hi = b - 1;
        bool found = false;
        while (lo <= hi && !found) {
            const int mid = (lo + hi) >> 1, v = cl_idx[mid];
            found = v == I;
            if (v < I) lo = mid + 1; else hi = mid - 1;
        }
        missing += found ? 0 : 1;
    }
    if (missing) atomicAdd(count, missing);
}

void pattern_outside_clusters(int n, const int* row_ptr, const int* col_idx, const int* cl_ptr,
                              const int* cl_idx, int* count, cudaStream_t st) {
    const int T = 256;
    k_pattern_outside<<<(n + T - 1) / T, T, 0, st>>>(n, row_ptr, col_idx, cl_ptr, cl_idx, count);
}

}  // namespace elses
