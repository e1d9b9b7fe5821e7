// a7: chemical potential by bisection; a9: N(mu), E_band, Omega at a given mu.
//
// With the poles e_k and weights of every column, the electron count is
//     N(mu) = Tr(rho S) = sum_j sum_k 2 f(e_k - mu) d_k c_k,   f(x) = 1 / (1 + exp(x / kT)),
// and mu is found by bisection on N(mu) = N_e once G has been computed the first time (Eq. 3
// and the text after it). Reading: bracket [min e - 40 kT, max e + 40 kT]; each step replaces lo by mid
// when N(mid) < N_e, else hi; stop when hi - lo < tol or after max_iter steps; mu = (lo+hi)/2.
// E_band = sum 2 f g c = Tr(rho H) (Eq. 6); Omega = sum d c w(e), w = -2 kT ln(1 + e^{-(e-mu)/kT}).
//
// Once the bracket is narrower than 10 kT, the bisection step at its midpoint mu0 also keeps the
// poles within 60 kT of mu0 as E_k = exp((e_k - mu0)/kT) with their weight d_k c_k, compacted
// per block in pole order, and the sum of 2 d_k c_k of the poles below that window (when buffers
// are given). Every later midpoint x lies within 5 kT of mu0, so a kept pole has
// f = 1 / (1 + E_k exp((mu0 - x)/kT)), one exponential per launch instead of one per pole, a pole
// under the window has f = 1 and one above it f = 0 (to e^-55 of its weight, far under the
// rounding of the sums); the later steps read only the kept poles.
//
// Every evaluation is one grid-wide reduction in a fixed order (per-thread column strides, a
// fixed block tree, then the block partials summed in index order by the last block to finish,
// found with an atomic ticket -- no thread ever waits on another block). The bracket lives in
// device memory and each bisection launch reads and updates it, so the whole search is a fixed
// sequence of launches with no host round trip; launches after convergence return at once.
#include "internal.h"

namespace elses {

constexpr int kRedThreads = 256;

int reduce_grid() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 4 * (sms > 0 ? sms : 1);
}

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* partials, int nv_stride) {
    __shared__ double sh[NV][kRedThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = warp_sum(v[q]);
        if (lane == 0) sh[q][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int i = 0; i < kRedThreads / 32; ++i) s += sh[q][i];
            partials[(size_t)blockIdx.x * nv_stride + q] = s;
        }
    }
    __syncthreads();   // sh is read by thread 0 above: a later call must not overwrite it first
}

// True in every thread of the last block to finish (after all partials are visible).
__device__ __forceinline__ bool last_block(unsigned* ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    return is_last;
}

// Sum of the block partials [b][q], q < NV, by all threads of one block in a fixed order
// (thread t takes blocks t, t + T, ...; then a fixed tree). Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, int nblocks, double (&out)[NV]) {
    __shared__ double sh[NV][kRedThreads / 32];
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] += __ldcg(partials + 4 * (size_t)b + q);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double x = warp_sum(v[q]);
        if (lane == 0) sh[q][w] = x;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = 0.0;
        for (int i = 0; i < kRedThreads / 32; ++i) s += sh[q][i];
        out[q] = s;
    }
}

__global__ void k_bracket(const ReduceArgs a) {
    double mn = 1e300, mx = -1e300;
    const size_t total = (size_t)a.M * a.nu_max;   // one thread per pole slot (coalesced)
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(p / a.nu_max), k = (int)(p - (size_t)j * a.nu_max);
        if (k >= __ldg(a.nu_eff + j)) continue;
        const double e = a.eps[p];
        mn = fmin(mn, e);
        mx = fmax(mx, e);
    }
    __shared__ double smn[kRedThreads], smx[kRedThreads];
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.partials[4 * (size_t)blockIdx.x] = smn[0];
        a.partials[4 * (size_t)blockIdx.x + 1] = smx[0];
    }
    if (!last_block(a.ticket)) return;
    // the last block: the block extrema by all its threads (strided), then a tree
    double lo = 1e300, hi = -1e300;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        lo = fmin(lo, __ldcg(a.partials + 4 * (size_t)b));
        hi = fmax(hi, __ldcg(a.partials + 4 * (size_t)b + 1));
    }
    __syncthreads();   // smn / smx are reused
    smn[threadIdx.x] = lo;
    smx[threadIdx.x] = hi;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lo = smn[0];
        hi = smx[0];
        BisectState* s = a.state;
        s->lo = lo - 40.0 * a.kT;
        s->hi = hi + 40.0 * a.kT;
        s->iter = 0;
        s->done = (a.max_iter <= 0) || !(s->hi - s->lo >= a.tol);
        s->status = (lo <= hi && isfinite(lo) && isfinite(hi)) ? 0 : DEV_NONFINITE;
        s->mu = 0.5 * (s->lo + s->hi);
        s->mu0 = 0.0;
        s->have_pre = 0;
        *a.ticket = 0u;
    }
}

// mode 0: N(lo); 1: N(hi) and the bracket check; 2: one bisection step; 3: scalars at mu_in;
// 4: scalars at the state's mu (written like mode 3).
// Block b takes the poles of a contiguous range (flattened [column][k]); poles more than 50 kT
// from x contribute their limit (f = 1 below, 0 above) without an exponential: the neglected part
// is below e^-50 of their weight, far under the rounding of the sums.
__global__ void __launch_bounds__(kRedThreads) k_count(const ReduceArgs a, int mode, double mu_in) {
    BisectState* s = a.state;
    double x;
    if (mode == 2) {
        if (s->done) return;
        x = 0.5 * (s->lo + s->hi);
    } else if (mode == 0) x = s->lo;
    else if (mode == 1) x = s->hi;
    else if (mode == 4) x = s->mu;
    else x = mu_in;
    if (mode == 4) mode = 3;
    double v[3] = {0.0, 0.0, 0.0};
    const size_t total = (size_t)a.M * a.nu_max;
    const size_t chunk = (total + gridDim.x - 1) / gridDim.x;
    const size_t b0 = min(total, (size_t)blockIdx.x * chunk), b1 = min(total, b0 + chunk);
    const double inv_kT = a.inv_kT;
    const bool keep = mode == 2 && a.act && !s->have_pre && s->hi - s->lo < 10.0 * a.kT;
    if (mode == 2 && a.act && s->have_pre) {
        // the kept poles of this block; the block's constant part once, by thread 0
        const double scale = s->scale;   // exp((mu0 - x)/kT), set by the previous step
        const int n = a.act_n[blockIdx.x];
        const double2* q = a.act + b0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double2 w = q[i];
            v[0] = fma(2.0 / fma(w.x, scale, 1.0), w.y, v[0]);
        }
        if (threadIdx.x == 0) v[0] += a.act_below[blockIdx.x];
    } else {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        __shared__ int wcount[kRedThreads / 32];
        // the poles within 50 kT of x need exponentials; they wait in a per-warp buffer and are
        // evaluated 32 at a time with every lane busy (the FP64 pipe charges a warp instruction
        // whatever its active lanes), the others add their limits at once
        __shared__ double qt[kRedThreads / 32][64], qdc[kRedThreads / 32][64], qe[kRedThreads / 32][64],
            qg[kRedThreads / 32][64], qc[kRedThreads / 32][64];
        int nq = 0;
        auto evaluate = [&](int cnt) {
            if (lane < cnt) {
                const double t = qt[wid][lane], dc = qdc[wid][lane];
                const double f2 = 2.0 * fermi(t);
                v[0] = fma(f2, dc, v[0]);
                if (mode == 3) {
                    v[1] = fma(f2 * qg[wid][lane], qc[wid][lane], v[1]);
                    v[2] = fma(dc, omega_w(qe[wid][lane], x, a.kT), v[2]);
                }
            }
        };
        double below = 0.0;
        int kept = 0;
        for (size_t t0 = b0; t0 < b1; t0 += blockDim.x) {
            const size_t p = t0 + threadIdx.x;
            bool in_window = false, near = false;
            double Ek = 0.0, dcw = 0.0, t = 0.0, dc = 0.0, e = 0.0, cc = 0.0;
            if (p < b1) {
                const int j = (int)(p / a.nu_max), k = (int)(p - (size_t)j * a.nu_max);
                if (k < __ldg(a.nu_eff + j)) {
                    e = a.eps[p];
                    cc = a.c[p];
                    t = (e - x) * inv_kT;
                    dc = a.d[p] * cc;
                    if (keep) {
                        if (fabs(t) <= 60.0) {
                            in_window = true;
                            Ek = exp(t);
                            dcw = dc;
                        } else if (t < -60.0) {
                            below = fma(2.0, dc, below);
                        }
                    }
                    if (t < -50.0) {          // f = 1, w = 2 (e - x) to e^-50 of the weight
                        v[0] = fma(2.0, dc, v[0]);
                        if (mode == 3) {
                            v[1] = fma(2.0 * a.g[p], cc, v[1]);
                            v[2] = fma(dc, 2.0 * (e - x), v[2]);
                        }
                    } else if (t <= 50.0) {
                        near = true;
                    }
                }
            }
            {   // buffer this tile's near poles; evaluate a full buffer
                const unsigned m = __ballot_sync(0xffffffffu, near);
                if (near) {
                    const int q = nq + __popc(m & ((1u << lane) - 1u));
                    qt[wid][q] = t;
                    qdc[wid][q] = dc;
                    if (mode == 3) {
                        qe[wid][q] = e;
                        qg[wid][q] = a.g[p];
                        qc[wid][q] = cc;
                    }
                }
                nq += __popc(m);
                __syncwarp();
                if (nq >= 32) {
                    evaluate(32);
                    const int rest = nq - 32;
                    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0;
                    if (lane < rest) {
                        r0 = qt[wid][32 + lane];
                        r1 = qdc[wid][32 + lane];
                        if (mode == 3) {
                            r2 = qe[wid][32 + lane];
                            r3 = qg[wid][32 + lane];
                            r4 = qc[wid][32 + lane];
                        }
                    }
                    __syncwarp();
                    if (lane < rest) {
                        qt[wid][lane] = r0;
                        qdc[wid][lane] = r1;
                        if (mode == 3) {
                            qe[wid][lane] = r2;
                            qg[wid][lane] = r3;
                            qc[wid][lane] = r4;
                        }
                    }
                    nq = rest;
                    __syncwarp();
                }
            }
            if (keep) {   // this tile's kept poles, appended in pole order
                const unsigned m = __ballot_sync(0xffffffffu, in_window);
                if (lane == 0) wcount[wid] = __popc(m);
                __syncthreads();
                int off = kept, tot = kept;
                for (int q = 0; q < kRedThreads / 32; ++q) {
                    if (q < wid) off += wcount[q];
                    tot += wcount[q];
                }
                if (in_window) a.act[b0 + off + __popc(m & ((1u << lane) - 1u))] = make_double2(Ek, dcw);
                __syncthreads();
                kept = tot;
            }
        }
        if (nq > 0) evaluate(nq);
        if (keep) {
            double bl[1] = {below};
            block_reduce_store<1>(bl, a.act_below, 1);
            if (threadIdx.x == 0) a.act_n[blockIdx.x] = kept;
        }
    }
    // the bisection needs N only; mode 3 also E_band and Omega
    if (mode == 3) block_reduce_store<3>(v, a.partials, 4);
    else {
        double n1[1] = {v[0]};
        block_reduce_store<1>(n1, a.partials, 4);
    }
    if (!last_block(a.ticket)) return;
    double tot[3] = {0.0, 0.0, 0.0};
    if (mode == 3) sum_partials<3>(a.partials, gridDim.x, tot);
    else {
        double t1[1];
        sum_partials<1>(a.partials, gridDim.x, t1);
        tot[0] = t1[0];
    }
    if (threadIdx.x == 0) {
        const double N = tot[0], E = tot[1], Om = tot[2];
        if (mode == 0) s->n_lo = N;
        else if (mode == 1) {
            s->n_hi = N;
            if (!(s->n_lo < a.n_electrons && a.n_electrons <= N)) {
                s->status |= DEV_NO_BRACKET;
                s->done = 1;
            }
        } else if (mode == 2) {
            if (keep) {
                s->have_pre = 1;
                s->mu0 = x;
            }
            if (N < a.n_electrons) s->lo = x; else s->hi = x;
            s->n_mid = N;
            s->iter += 1;
            if (s->iter >= a.max_iter || !(s->hi - s->lo >= a.tol)) s->done = 1;
            s->mu = 0.5 * (s->lo + s->hi);
            if (s->have_pre) s->scale = exp((s->mu0 - 0.5 * (s->lo + s->hi)) * inv_kT);
        } else {
            s->n_at = N;
            s->e_band = E;
            s->omega = Om;
        }
        *a.ticket = 0u;
    }
}

void bisect_init(const ReduceArgs& a, cudaStream_t st) {
    const int G = reduce_grid();
    k_bracket<<<G, kRedThreads, 0, st>>>(a);
    k_count<<<G, kRedThreads, 0, st>>>(a, 0, 0.0);
    k_count<<<G, kRedThreads, 0, st>>>(a, 1, 0.0);
}

void bisect_step(const ReduceArgs& a, cudaStream_t st) {
    k_count<<<reduce_grid(), kRedThreads, 0, st>>>(a, 2, 0.0);
}

void scalars_at(const ReduceArgs& a, double mu, cudaStream_t st) {
    k_count<<<reduce_grid(), kRedThreads, 0, st>>>(a, 3, mu);
}

void scalars_at_state(const ReduceArgs& a, cudaStream_t st) {
    k_count<<<reduce_grid(), kRedThreads, 0, st>>>(a, 4, 0.0);
}

// Density of states -(1/pi) Im sum_j sum_k d_k c_k / (z - e_k) at the energies z[iz] (grid
// (blocks, n_z)): per block a fixed-order tree into partials[iz][block]; k_dos_sum then adds the
// blocks in index order, so the result does not depend on the order in which blocks finish.
__global__ void __launch_bounds__(kRedThreads) k_dos(const ReduceArgs a, const double* __restrict__ z,
                                                     double* partials) {
    const int iz = blockIdx.y;
    const double zr = z[2 * iz], zi = z[2 * iz + 1];
    const size_t total = (size_t)a.M * a.nu_max;
    double v = 0.0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(p / a.nu_max), k = (int)(p - (size_t)j * a.nu_max);
        if (k >= __ldg(a.nu_eff + j)) continue;
        const double dr = zr - a.eps[p];
        v = fma(a.d[p] * a.c[p], zi / fma(dr, dr, zi * zi), v);    // -Im 1/(z - e) = zi / |z - e|^2
    }
    __shared__ double sv[kRedThreads];
    sv[threadIdx.x] = v;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sv[threadIdx.x] += sv[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[(size_t)iz * gridDim.x + blockIdx.x] = sv[0];
}

__global__ void __launch_bounds__(kRedThreads) k_dos_sum(const double* __restrict__ partials, int nblocks,
                                                         double* out) {
    const int iz = blockIdx.x;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(size_t)iz * nblocks + b];
    __shared__ double sv[kRedThreads];
    sv[threadIdx.x] = v;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sv[threadIdx.x] += sv[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[iz] = sv[0] * 0.31830988618379067154;
}

size_t dos_scratch_doubles(int n_z) { return (size_t)n_z * (reduce_grid() + 1); }

void dos_at(const ReduceArgs& a, const double* z_dev, int n_z, double* scratch, cudaStream_t st) {
    const int G = reduce_grid();
    k_dos<<<dim3(G, n_z), kRedThreads, 0, st>>>(a, z_dev, scratch);
    k_dos_sum<<<n_z, kRedThreads, 0, st>>>(scratch, G, scratch + (size_t)n_z * G);
}

}  // namespace elses
