// Device building blocks shared by the Krylov kernel (a3 + a4, krylov.cu) and the adjoint
// kernel (adjoint.cu): the per-lane entry lists of a cluster, the sparse products, the CGS
// helpers and the forward Krylov recursion of one column.
//
// Layout (one CTA of 4 warps per atom J, one warp per orbital column alpha): the cluster's atoms
// are sorted by in-cluster degree and dealt to the lanes with the shortest lists, so that
// lane work is balanced; each lane owns whole atoms (4 rows). A vector of the cluster is held
// in "position" order: position p = slot * 32 + lane, orbital r at 4 p + r. The bases live in
// global scratch as [k][position][orbital] (coalesced 32-byte rows per lane). The forms ending in
// _w at the end of the file do the same for groups of W lanes per column.
#pragma once

#include "internal.h"

namespace elses {

struct __align__(8) Ent {
    int p4;   // 4 * (lane-slot position of the neighbour atom) = offset into a shared vector
    int blk;  // BSR block index, -1 = padding
};

constexpr int kThreads = 32 * kWarpsPerAtom;

__device__ __forceinline__ int bsearch_sorted(const int* a, int n, int v) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int x = a[mid];
        if (x == v) return mid;
        if (x < v) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__device__ __forceinline__ int nu_for(const KrylovArgs& a, int n_at) {
    for (int c = 0; c < a.n_classes; ++c)
        if (n_at <= a.class_max_atoms[c]) return a.class_nu[c];
    return a.nu_default;
}

// acc + a . b over 4 orbitals: four FMAs straight into the accumulator.
__device__ __forceinline__ double fma4(const double2 a0, const double2 a1, const double2 b0, const double2 b1,
                                       double acc) {
    return fma(a1.y, b1.y, fma(a1.x, b1.x, fma(a0.y, b0.y, fma(a0.x, b0.x, acc))));
}

// y = A x on the cluster (lane-owned rows; x gathered from shared memory, y in shared or global
// memory). Each lane walks one list holding the entries of all its rows in slot order
// (entry.p4 low 16 bits: neighbour offset in x; high bits: the row's slot), so lanes stop after
// their own entry count instead of after the widest row of every slot. Rows start from the
// on-site term: the diagonal of the on-site block of `dvals` (block index eself[p]), the
// identity when dvals is null, or zero when the on-site block is a list entry. With `skr` the
// off-site blocks are applied in their two-centre form (13 FP64 instructions instead of 16;
// which = 0 selects the H integrals, 1 the S integrals).
__device__ __forceinline__ void spmv(const double* __restrict__ vals, const double* __restrict__ skr,
                                     int which, const Ent* __restrict__ ent, int kmax, int NS,
                                     const double* x, double* y, int lane, bool onsite,
                                     const double* __restrict__ dvals, const int* eself) {
    for (int s = 0; s < NS; ++s) {
        const int p = s * 32 + lane, po = 4 * p;
        double2 o01 = make_double2(0.0, 0.0), o23 = make_double2(0.0, 0.0);
        if (onsite) {
            o01 = *reinterpret_cast<const double2*>(x + po);
            o23 = *reinterpret_cast<const double2*>(x + po + 2);
            const int es = eself[p];
            if (dvals && es >= 0) {
                const double* d = dvals + 16 * (size_t)es;
                o01.x *= __ldg(d); o01.y *= __ldg(d + 5); o23.x *= __ldg(d + 10); o23.y *= __ldg(d + 15);
            }
        }
        *reinterpret_cast<double2*>(y + po) = o01;
        *reinterpret_cast<double2*>(y + po + 2) = o23;
    }
    int cur = -1;
    double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
    for (int k = 0; k < kmax; ++k) {
        const Ent en = ent[32 * k + lane];
        if (en.blk >= 0) {
            const int s = en.p4 >> 16, p4 = en.p4 & 0xffff;
            if (s != cur) {
                if (cur >= 0) {
                    double2* yo = reinterpret_cast<double2*>(y + 4 * (cur * 32 + lane));
                    yo[0] = make_double2(y0, y1);
                    yo[1] = make_double2(y2, y3);
                }
                cur = s;
                const double2* yi = reinterpret_cast<const double2*>(y + 4 * (s * 32 + lane));
                const double2 i01 = yi[0], i23 = yi[1];
                y0 = i01.x; y1 = i01.y; y2 = i23.x; y3 = i23.y;
            }
            const double2 x01 = *reinterpret_cast<const double2*>(x + p4);
            const double2 x23 = *reinterpret_cast<const double2*>(x + p4 + 2);
            if (skr) {
                // two-centre block: t = u.x_p; y_s += V_ss x_s + V_sp t;
                // y_p += V_pi x_p + (dV t - V_sp x_s) u,  dV = V_pp_sigma - V_pp_pi
                const double2* q = reinterpret_cast<const double2*>(skr + 12 * (size_t)en.blk);
                const double2 u01 = __ldg(q), u2_ = __ldg(q + 1);
                const double2 v01 = __ldg(q + 2 + 2 * which), v23 = __ldg(q + 3 + 2 * which);
                const double t = fma(u2_.x, x23.y, fma(u01.y, x23.x, u01.x * x01.y));
                y0 = fma(v01.y, t, fma(v01.x, x01.x, y0));
                const double aa = fma(v23.y, t, -v01.y * x01.x);
                y1 = fma(aa, u01.x, fma(v23.x, x01.y, y1));
                y2 = fma(aa, u01.y, fma(v23.x, x23.x, y2));
                y3 = fma(aa, u2_.x, fma(v23.x, x23.y, y3));
            } else {
                const double2* b2 = reinterpret_cast<const double2*>(vals + 16 * (size_t)en.blk);
                const double2 a0 = __ldg(b2 + 0), a1 = __ldg(b2 + 1), a2 = __ldg(b2 + 2), a3 = __ldg(b2 + 3);
                const double2 a4 = __ldg(b2 + 4), a5 = __ldg(b2 + 5), a6 = __ldg(b2 + 6), a7 = __ldg(b2 + 7);
                y0 = fma(a0.x, x01.x, fma(a0.y, x01.y, fma(a1.x, x23.x, fma(a1.y, x23.y, y0))));
                y1 = fma(a2.x, x01.x, fma(a2.y, x01.y, fma(a3.x, x23.x, fma(a3.y, x23.y, y1))));
                y2 = fma(a4.x, x01.x, fma(a4.y, x01.y, fma(a5.x, x23.x, fma(a5.y, x23.y, y2))));
                y3 = fma(a6.x, x01.x, fma(a6.y, x01.y, fma(a7.x, x23.x, fma(a7.y, x23.y, y3))));
            }
        }
    }
    if (cur >= 0) {
        double2* yo = reinterpret_cast<double2*>(y + 4 * (cur * 32 + lane));
        yo[0] = make_double2(y0, y1);
        yo[1] = make_double2(y2, y3);
    }
}

__device__ __forceinline__ void ld4(const double* p, double2& a, double2& b) {
    const double2* q = reinterpret_cast<const double2*>(p);
    a = q[0];
    b = q[1];
}
__device__ __forceinline__ void st4(double* p, const double2 a, const double2 b) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = a;
    q[1] = b;
}

// Hint that the 32-byte row at p be brought into L2 (no register, no wait; in-bounds addresses
// only), so that a later load finds it there instead of in DRAM.
__device__ __forceinline__ void prefetch_l2(const double* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// w -= sum_{k <= n} U[:, k] h_k on the lane's rows of slot position p; the basis rows are
// fetched four at a time before they are used, so their latency overlaps, and the rows of the
// next position pn (pn < 0: none) are prefetched into L2 beside them. (Four at a time: 87.4 ms
// for the 4096-atom Krylov phase, against 89.7 with six and 93.4 with eight, whose registers
// spill; two and three do as well as four.)
__device__ __forceinline__ void sub_basis(const double* Ub, int NP, int p, const double* h, int n,
                                          double2& w0, double2& w1, int pn = -1) {
    for (int k0 = 0; k0 <= n; k0 += 4) {
        double2 ua[4], ub[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            if (k0 + kk <= n) {
                ld4(Ub + 4 * ((size_t)(k0 + kk) * NP + p), ua[kk], ub[kk]);
                if (pn >= 0) prefetch_l2(Ub + 4 * ((size_t)(k0 + kk) * NP + pn));
            }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            if (k0 + kk <= n) {
                const double hk = h[k0 + kk];
                w0.x = fma(-ua[kk].x, hk, w0.x);
                w0.y = fma(-ua[kk].y, hk, w0.y);
                w1.x = fma(-ub[kk].x, hk, w1.x);
                w1.y = fma(-ub[kk].y, hk, w1.y);
            }
        }
    }
}

// y_H = H x and y_S = S x in one pass over the lane's list entries (x gathered once per entry for
// both; in the two-centre form the projection t = u . x_p is shared by the H and S blocks, 23
// FP64 instructions per entry instead of 2 x 13). Each product is the one spmv_w forms, bit for
// bit: y_H with the diagonal of H's on-site block, y_S with the identity on-site (Slater-Koster
// systems), or both with the on-site blocks as list entries. yH and yS may be shared or global.
template <int W>
__device__ __forceinline__ void spmv_hs_w(const double* __restrict__ Hv, const double* __restrict__ Sv,
                                          const double* __restrict__ skr, const Ent* __restrict__ ent,
                                          int kmax, int NS, const double* x, double* yH, double* yS,
                                          int lane, bool onsite, const int* eself) {
    for (int s = 0; s < NS; ++s) {
        const int p = s * W + lane, po = 4 * p;
        double2 h01 = make_double2(0.0, 0.0), h23 = h01, s01 = h01, s23 = h01;
        if (onsite) {
            s01 = *reinterpret_cast<const double2*>(x + po);
            s23 = *reinterpret_cast<const double2*>(x + po + 2);
            h01 = s01;
            h23 = s23;
            const int es = eself[p];
            if (es >= 0) {
                const double* d = Hv + 16 * (size_t)es;
                h01.x *= __ldg(d); h01.y *= __ldg(d + 5); h23.x *= __ldg(d + 10); h23.y *= __ldg(d + 15);
            }
        }
        st4(yH + po, h01, h23);
        st4(yS + po, s01, s23);
    }
    int cur = -1;
    double h0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int k = 0; k < kmax; ++k) {
        const Ent en = ent[W * k + lane];
        if (en.blk >= 0) {
            const int sl = en.p4 >> 16, p4 = en.p4 & 0xffff;
            if (sl != cur) {
                if (cur >= 0) {
                    const int po = 4 * (cur * W + lane);
                    st4(yH + po, make_double2(h0, h1), make_double2(h2, h3));
                    st4(yS + po, make_double2(s0, s1), make_double2(s2, s3));
                }
                cur = sl;
                const int po = 4 * (sl * W + lane);
                double2 a, b;
                ld4(yH + po, a, b);
                h0 = a.x; h1 = a.y; h2 = b.x; h3 = b.y;
                ld4(yS + po, a, b);
                s0 = a.x; s1 = a.y; s2 = b.x; s3 = b.y;
            }
            const double2 x01 = *reinterpret_cast<const double2*>(x + p4);
            const double2 x23 = *reinterpret_cast<const double2*>(x + p4 + 2);
            if (skr) {
                // two-centre blocks (as in spmv_w): t = u.x_p; y_s += V_ss x_s + V_sp t;
                // y_p += V_pi x_p + (dV t - V_sp x_s) u, with the H and the S integrals
                const double2* q = reinterpret_cast<const double2*>(skr + 12 * (size_t)en.blk);
                const double2 u01 = __ldg(q), u2_ = __ldg(q + 1);
                const double2 a01 = __ldg(q + 2), a23 = __ldg(q + 3), b01 = __ldg(q + 4), b23 = __ldg(q + 5);
                const double t = fma(u2_.x, x23.y, fma(u01.y, x23.x, u01.x * x01.y));
                h0 = fma(a01.y, t, fma(a01.x, x01.x, h0));
                const double ah = fma(a23.y, t, -a01.y * x01.x);
                h1 = fma(ah, u01.x, fma(a23.x, x01.y, h1));
                h2 = fma(ah, u01.y, fma(a23.x, x23.x, h2));
                h3 = fma(ah, u2_.x, fma(a23.x, x23.y, h3));
                s0 = fma(b01.y, t, fma(b01.x, x01.x, s0));
                const double as = fma(b23.y, t, -b01.y * x01.x);
                s1 = fma(as, u01.x, fma(b23.x, x01.y, s1));
                s2 = fma(as, u01.y, fma(b23.x, x23.x, s2));
                s3 = fma(as, u2_.x, fma(b23.x, x23.y, s3));
            } else {
                const double2* bh = reinterpret_cast<const double2*>(Hv + 16 * (size_t)en.blk);
                const double2* bs = reinterpret_cast<const double2*>(Sv + 16 * (size_t)en.blk);
                double2 c0 = __ldg(bh + 0), c1 = __ldg(bh + 1), c2 = __ldg(bh + 2), c3 = __ldg(bh + 3);
                double2 c4 = __ldg(bh + 4), c5 = __ldg(bh + 5), c6 = __ldg(bh + 6), c7 = __ldg(bh + 7);
                h0 = fma(c0.x, x01.x, fma(c0.y, x01.y, fma(c1.x, x23.x, fma(c1.y, x23.y, h0))));
                h1 = fma(c2.x, x01.x, fma(c2.y, x01.y, fma(c3.x, x23.x, fma(c3.y, x23.y, h1))));
                h2 = fma(c4.x, x01.x, fma(c4.y, x01.y, fma(c5.x, x23.x, fma(c5.y, x23.y, h2))));
                h3 = fma(c6.x, x01.x, fma(c6.y, x01.y, fma(c7.x, x23.x, fma(c7.y, x23.y, h3))));
                c0 = __ldg(bs + 0); c1 = __ldg(bs + 1); c2 = __ldg(bs + 2); c3 = __ldg(bs + 3);
                c4 = __ldg(bs + 4); c5 = __ldg(bs + 5); c6 = __ldg(bs + 6); c7 = __ldg(bs + 7);
                s0 = fma(c0.x, x01.x, fma(c0.y, x01.y, fma(c1.x, x23.x, fma(c1.y, x23.y, s0))));
                s1 = fma(c2.x, x01.x, fma(c2.y, x01.y, fma(c3.x, x23.x, fma(c3.y, x23.y, s1))));
                s2 = fma(c4.x, x01.x, fma(c4.y, x01.y, fma(c5.x, x23.x, fma(c5.y, x23.y, s2))));
                s3 = fma(c6.x, x01.x, fma(c6.y, x01.y, fma(c7.x, x23.x, fma(c7.y, x23.y, s3))));
            }
        }
    }
    if (cur >= 0) {
        const int po = 4 * (cur * W + lane);
        st4(yH + po, make_double2(h0, h1), make_double2(h2, h3));
        st4(yS + po, make_double2(s0, s1), make_double2(s2, s3));
    }
}

// Sum of 16 values held by every lane over the 32 lanes (recursive halving on lane bits 3..0,
// then one exchange across bit 4): lanes l and l + 16 end with the sum of value l & 15.
__device__ __forceinline__ double warp_sum16(double (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            double send = upper ? v[i] : v[i + w];
            double keep = upper ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// Shared-memory view of the cluster of one atom: its atoms (sorted), their in-cluster degrees,
// the lane-slot position of each and the per-lane entry lists.
struct ClusterView {
    Ent* ell;             // [kmax][32] entry lists, lane-interleaved
    int* cl;              // cluster atoms, ascending
    int* deg;             // in-cluster list length of each cluster atom
    int* pos_of;          // position of each cluster atom
    int* atom_at;         // cluster atom at each position (-1: empty)
    int* eoff;            // first list entry of each position
    int* eself;           // on-site block of each position (-1: none)
    int n_at, NS, kmax, nent;
};

__host__ __device__ inline size_t view_bytes(int NA, int deg_max) {
    return sizeof(Ent) * (size_t)NA * deg_max + sizeof(int) * (size_t)(6 * NA + 2);
}

__device__ __forceinline__ void carve_view(unsigned char* base, int NA, int deg_max, ClusterView& v) {
    v.ell = reinterpret_cast<Ent*>(base);
    v.cl = reinterpret_cast<int*>(v.ell + (size_t)NA * deg_max);
    v.deg = v.cl + NA;
    v.pos_of = v.deg + NA;
    v.atom_at = v.pos_of + NA;
    v.eoff = v.atom_at + NA;
    v.eself = v.eoff + NA;
}

// Positions of the cluster atoms (W lanes, NS slots each; every thread of the CTA's T calls).
// The lanes' list lengths set the trip count of the sparse products, so they are balanced. The
// atoms go in decreasing in-cluster degree (ties by index) one at a time to the lane whose list
// is shortest so far among the lanes with a free slot (ties to the lowest lane), into its next
// slot. Then, while the longest list can be shortened by moving one of its atoms to a free slot
// of another lane or by swapping it for an atom of lower degree there, the change that shortens
// it most is made (ties: lowest lane, then lowest slots; at most 64 changes). On 6 A diamond
// clusters the longest list ends 1.1% above the mean, at the bound ceil(total / W) (2.8% after
// the first pass alone, 7% for a snake order over degree-sorted atoms). `atom_at` serves as
// scratch for the atoms in rank order, then holds the atom at each position (-1: empty).
template <int W, int T>
__device__ __forceinline__ void balanced_positions(int n_at, int NS, const int* deg, int* pos_of, int* atom_at) {
    const int tid = threadIdx.x;
    for (int q = tid; q < n_at; q += T) {
        const int dq = deg[q];
        int rank = 0;
        for (int b = 0; b < n_at; ++b) {
            const int db = deg[b];
            rank += (db > dq) || (db == dq && b < q);
        }
        atom_at[rank] = q;
    }
    __syncthreads();
    if (tid < W) {
        const unsigned m = W == 32 ? 0xffffffffu : 0xffffu;
        int tot = 0, cnt = 0;
        for (int r = 0; r < n_at; ++r) {
            const int q = atom_at[r];
            int key = cnt < NS ? tot * W + tid : 0x7fffffff;
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(m, key, o));
            if (key % W == tid) {
                pos_of[q] = cnt * W + tid;
                ++cnt;
                tot += deg[q];
            }
        }
    }
    __syncthreads();
    for (int p = tid; p < NS * W; p += T) atom_at[p] = -1;
    __syncthreads();
    for (int q = tid; q < n_at; q += T) atom_at[pos_of[q]] = q;
    __syncthreads();
    if (tid < W) {
        const unsigned m = W == 32 ? 0xffffffffu : 0xffffu;
        int tot = 0;
        for (int sl = 0; sl < NS; ++sl) {
            const int q = atom_at[sl * W + tid];
            if (q >= 0) tot += deg[q];
        }
        for (int it = 0; it < 64; ++it) {
            int key = tot * W + (W - 1 - tid);       // the longest list, ties to the lowest lane
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(m, key, o));
            const int Lm = W - 1 - key % W, tmax = key / W;
            int best = 0;                            // gain << 16 | (63 - slot a) << 8 | (63 - slot b)
            if (tid != Lm) {
                for (int sa = 0; sa < NS; ++sa) {
                    const int qa = atom_at[sa * W + Lm];
                    if (qa < 0) continue;
                    const int da = deg[qa];
                    for (int sb = 0; sb < NS; ++sb) {
                        const int qb = atom_at[sb * W + tid];
                        const int d = da - (qb >= 0 ? deg[qb] : 0);   // qb < 0: a move to a free slot
                        if (d <= 0) continue;
                        const int gain = tmax - max(tmax - d, tot + d);
                        if (gain > 0) best = max(best, (gain << 16) | ((63 - sa) << 8) | (63 - sb));
                    }
                }
            }
            int bmax = best;
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) bmax = max(bmax, __shfl_xor_sync(m, bmax, o));
            if (bmax <= 0) break;
            int L2 = best == bmax ? tid : W;          // ties to the lowest lane
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) L2 = min(L2, __shfl_xor_sync(m, L2, o));
            const int sa = 63 - ((bmax >> 8) & 255), sb = 63 - (bmax & 255);
            const int qa = atom_at[sa * W + Lm], qb = atom_at[sb * W + L2];
            const int d = deg[qa] - (qb >= 0 ? deg[qb] : 0);
            __syncwarp(m);                           // every lane has read the old positions
            if (tid == L2) {
                atom_at[sa * W + Lm] = qb;
                atom_at[sb * W + L2] = qa;
                pos_of[qa] = sb * W + L2;
                if (qb >= 0) pos_of[qb] = sa * W + Lm;
            }
            if (tid == Lm) tot -= d;
            if (tid == L2) tot += d;
            __syncwarp(m);
        }
    }
    __syncthreads();
}

// Builds the view of atom J's cluster (every thread of the CTA calls it). Returns false, the
// same on every thread, when the cluster exceeds NA atoms or the lists exceed their capacity.
__device__ __forceinline__ bool cluster_view(const KrylovArgs& a, int J, int NA, ClusterView& v) {
    __shared__ int sh_bad, sh_kmax, sh_nent;
    const int tid = threadIdx.x;
    const bool onsite = a.onsite_diag != 0;
    Ent* ell = v.ell;
    int* cl = v.cl;
    int* deg = v.deg;
    int* pos_of = v.pos_of;
    int* atom_at = v.atom_at;
    int* eoff = v.eoff;
    int* eself = v.eself;
    int n_at, cbase = 0;
    if (a.cl_ptr) { cbase = a.cl_ptr[J]; n_at = a.cl_ptr[J + 1] - cbase; }
    else n_at = a.n_atoms;
    if (n_at > NA) return false;   // uniform across the CTA
    for (int q = tid; q < n_at; q += kThreads) cl[q] = a.cl_ptr ? a.cl_idx[cbase + q] : q;
    __syncthreads();
    for (int q = tid; q < n_at; q += kThreads) {
        const int A = cl[q];
        int cnt = 0;
        for (int e = a.row_ptr[A]; e < a.row_ptr[A + 1]; ++e) {
            const int ce = a.col_idx[e];
            cnt += (!onsite || ce != A) && bsearch_sorted(cl, n_at, ce) >= 0;
        }
        deg[q] = cnt;
    }
    __syncthreads();
    const int NS = (n_at + 31) >> 5;
    balanced_positions<32, kThreads>(n_at, NS, deg, pos_of, atom_at);
    // per-lane lists: the entries of the lane's rows in slot order
    if (tid < 32) {
        int off = 0;
        for (int sl = 0; sl < NS; ++sl) {
            const int pp = sl * 32 + tid;
            const int q = atom_at[pp];
            eoff[pp] = off;
            off += q >= 0 ? deg[q] : 0;
        }
        int kmax = off, ntot = off;
        for (int o = 16; o > 0; o >>= 1) {
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
            ntot += __shfl_xor_sync(0xffffffffu, ntot, o);
        }
        if (tid == 0) {
            sh_nent = ntot;
            sh_kmax = kmax;
            sh_bad = kmax * 32 > NA * a.deg_max;
        }
    }
    __syncthreads();
    if (sh_bad) return false;
    const int kmax = sh_kmax;
    for (int q = tid; q < kmax * 32; q += kThreads) ell[q] = Ent{0, -1};
    __syncthreads();
    for (int p = tid; p < NS * 32; p += kThreads) {
        const int q = atom_at[p];
        const int sl = p >> 5, l = p & 31;
        int k = eoff[p];
        int es = -1;
        if (q >= 0) {
            const int A = cl[q];
            for (int e = a.row_ptr[A]; e < a.row_ptr[A + 1]; ++e) {
                const int ce = a.col_idx[e];
                if (onsite && ce == A) {
                    es = e;
                    continue;
                }
                const int b = bsearch_sorted(cl, n_at, ce);
                if (b >= 0) ell[32 * (k++) + l] = Ent{(4 * pos_of[b]) | (sl << 16), e};
            }
        }
        eself[p] = es;
    }
    __syncthreads();
    v.n_at = n_at;
    v.NS = NS;
    v.kmax = kmax;
    v.nent = sh_nent;
    return true;
}

// Algorithmic FP64 flops of one column. Sparse products: nu_eff of H and S together, per
// off-site block 43 flops in the two-centre form (the projection t = u . x_p, 5 flops, shared by
// the two blocks of 19) or 64 as two dense blocks, the on-site H diagonal 4 per atom, the
// on-site S = I none. Dense work over the n_c = 4 n_at rows: per step n < nu_eff, pass A's three
// products and ||H u_n||^2, (6 (n+1) + 2) n_c; per step n < nu_eff - 1, the Gram-Schmidt
// updates and second-pass products, 6 (n+1) n_c with two classical passes or 2 (n+1) n_c +
// 2 (n+1)^2 with the second pass from S', then w^T S w and the scaling of u and S u, 4 n_c.
__device__ __forceinline__ unsigned long long column_flops(const KrylovArgs& a, int n_at, int nent, int nu_eff,
                                                           bool from_overlap) {
    const unsigned long long ne = (unsigned long long)nent, na = (unsigned long long)n_at;
    const unsigned long long nc = 4ull * na, vv = (unsigned long long)nu_eff;
    const unsigned long long pair = a.skr ? 43ull : 64ull;   // flops per block pair (H, S)
    const unsigned long long spm = a.onsite_diag ? vv * (pair * ne + 4ull * na) : vv * pair * ne;
    const unsigned long long tri = vv * (vv + 1) / 2;                 // sum_{n<v} (n+1)
    const unsigned long long trim = vv > 0 ? (vv - 1) * vv / 2 : 0;   // sum_{n<v-1} (n+1)
    const unsigned long long sq = vv > 0 ? (vv - 1) * vv * (2 * vv - 1) / 6 : 0;   // sum_{n<v-1} (n+1)^2
    unsigned long long dense = nc * (6 * tri + 2 * vv);
    if (vv > 0) dense += from_overlap ? nc * (2 * trim + 4 * (vv - 1)) + 2 * sq : nc * (6 * trim + 4 * (vv - 1));
    return spm + dense;
}

// The second Gram-Schmidt pass from the projected overlap (KrylovArgs::reorth = 1). With
// E = S' - I over k, q <= n (S' packed upper at sp, this step's column already written), the
// second pass's coefficients SU^T (w - U h) equal -E h in exact arithmetic, since SU^T U = S'.
// So h becomes h - E h, the coefficients of both passes together, and one sweep of the basis
// subtracts them. S'_kk - 1 is exact (S'_kk is within rounding of 1); the off-diagonal terms
// are summed first (the diagonal one selected away, no FP64 instruction) and the diagonal term
// added last. Lane l of the group of W lanes (mask m) forms the values k = l, l + W, ...; every
// lane must call.
template <int W>
__device__ __forceinline__ void second_pass_from_overlap(const double* __restrict__ sp, double* h, int n,
                                                        int lane, unsigned m) {
    constexpr int KR = kMaxNu / W;
    double g[KR];
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        const int k = lane + r * W;
        g[r] = 0.0;
        if (k <= n) {
            double eh = 0.0;
            for (int q = 0; q <= n; ++q) {
                const int lo = min(k, q), hi = max(k, q);
                const double e = q == k ? 0.0 : sp[lo + hi * (hi + 1) / 2];
                eh = fma(e, h[q], eh);
            }
            eh = fma(sp[k + k * (k + 1) / 2] - 1.0, h[k], eh);
            g[r] = h[k] - eh;
        }
    }
    __syncwarp(m);
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        const int k = lane + r * W;
        if (k <= n) h[k] = g[r];
    }
    __syncwarp(m);
}

// Forward Krylov recursion of column j = 4 J + alpha by one warp (the reading of the module
// header of krylov.cu): leaves U and SU in Uw, SUw ([k][position][orbital]) and writes H', S'
// (packed upper) and row j of U, SU, HU of the column. With kAdj it also keeps HU in HUw and the
// Gram-Schmidt coefficients in hess[n][k] (row stride nu_max): SU_k . HU_n for k <= n (the
// first pass) and beta_n at k = n + 1, which the adjoint needs. A and B are the warp's two
// shared vectors (u_1, then by turns H u_n -> w and the products H w of the next vector), h its
// coefficient buffer. The H and S products of each new vector are formed together from w
// (spmv_hs_w); the S product is scaled by 1 / beta with w, the H product is kept unscaled and its
// scale carried as a scalar (pscale). Returns nu_eff (nu_out: the column's nu), or 0
// for bad input (flagged).
template <bool kAdj>
__device__ __forceinline__ int column_forward(const KrylovArgs& a, const ClusterView& v, int J, int alpha,
                                              double* A, double* B, double* h, double* Uw, double* SUw,
                                              double* HUw, double* hess, int& nu_out, int& jp_out) {
    const int lane = threadIdx.x & 31;
    const bool onsite = a.onsite_diag != 0;
    const int n_at = v.n_at, NS = v.NS, kmax = v.kmax;
    const int* cl = v.cl;
    const int* pos_of = v.pos_of;
    const Ent* ell = v.ell;
    const int* eself = v.eself;
    const int PK = a.nu_max * (a.nu_max + 1) / 2;
    const int j = 4 * J + alpha;
    const int col = j - 4 * a.atom_begin;
    const int NP = NS * 32;
    const int nu = min(nu_for(a, n_at), a.nu_max);
    nu_out = nu;
    const int aJ = bsearch_sorted(cl, n_at, J);
    int eJJ = -1;
    for (int e = a.row_ptr[J]; e < a.row_ptr[J + 1]; ++e)
        if (a.col_idx[e] == J) eJJ = e;
    const double sjj = eJJ >= 0 ? a.S[16 * (size_t)eJJ + 5 * alpha] : -1.0;
    if (aJ < 0 || !(sjj > 0.0)) {   // no diagonal block or S_jj <= 0: bad input
        if (lane == 0) { flag(a.status, DEV_ARG); a.nu_eff[j] = 0; }
        return 0;
    }
    const int jp = 4 * pos_of[aJ] + alpha;
    jp_out = jp;
    const size_t vs = (size_t)NP * 4;                    // one basis vector

    for (int q = lane; q < NP * 4; q += 32) A[q] = 0.0;
    __syncwarp();
    if (lane == 0) A[jp] = 1.0 / sqrt(sjj);
    __syncwarp();
    // H u_1 -> B, S u_1 -> SU[0]; u_1 -> U[0]
    spmv_hs_w<32>(a.H, a.S, a.skr, ell, kmax, NS, A, B, SUw, lane, onsite, eself);
    for (int sl = 0; sl < NS; ++sl) {
        const int p = sl * 32 + lane;
        double2 x0, x1;
        ld4(A + 4 * p, x0, x1);
        st4(Uw + 4 * (size_t)p, x0, x1);
    }
    __syncwarp();

    // P holds H u_n at the top of step n (then w); the products of the next basis vector go to Q
    double* P = B;
    double* Q = A;
    // H u_n = pscale P: the H product of each new vector stays unscaled in P, and the values
    // formed from it (H', the first-pass coefficients) are scaled once as scalars
    double pscale = 1.0;
    int nu_eff = nu;
    for (int n = 0; n < nu; ++n) {
        double* SUn = SUw + (size_t)n * vs;
        if constexpr (kAdj) {
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * 32 + lane;
                double2 x0, x1;
                ld4(P + 4 * p, x0, x1);
                x0.x *= pscale; x0.y *= pscale; x1.x *= pscale; x1.y *= pscale;
                st4(HUw + (size_t)n * vs + 4 * p, x0, x1);
            }
        }
        if (lane == 0) {
            a.urow[(size_t)col * a.nu_max + n] = Uw[(size_t)n * vs + jp];
            a.surow[(size_t)col * a.nu_max + n] = SUn[jp];
            a.hurow[(size_t)col * a.nu_max + n] = P[jp] * pscale;
        }
        // pass A: H'[k][n], S'[k][n] and the first CGS coefficients, k <= n, five k at a time
        double hh = 0.0;
        for (int k0 = 0; k0 <= n; k0 += 5) {
            double acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.0;
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * 32 + lane;
                // the rows this chunk reads next: the next position, else the next chunk's first
                const int pn = sl + 1 < NS ? p + 32 : lane;
                const int kn = sl + 1 < NS ? k0 : k0 + 5;
                double2 hu0, hu1, su0, su1;
                ld4(P + 4 * p, hu0, hu1);
                ld4(SUn + 4 * p, su0, su1);
                if (k0 == 0) acc[15] = fma4(hu0, hu1, hu0, hu1, acc[15]);
#pragma unroll
                for (int kk = 0; kk < 5; ++kk) {
                    const int k = k0 + kk;
                    if (kn + kk <= n) {
                        prefetch_l2(Uw + (size_t)(kn + kk) * vs + 4 * pn);
                        prefetch_l2(SUw + (size_t)(kn + kk) * vs + 4 * pn);
                    }
                    if (k <= n) {
                        double2 u0, u1, v0, v1;
                        ld4(Uw + (size_t)k * vs + 4 * p, u0, u1);
                        ld4(SUw + (size_t)k * vs + 4 * p, v0, v1);
                        acc[kk] = fma4(u0, u1, hu0, hu1, acc[kk]);
                        acc[5 + kk] = fma4(u0, u1, su0, su1, acc[5 + kk]);
                        acc[10 + kk] = fma4(v0, v1, hu0, hu1, acc[10 + kk]);
                    }
                }
            }
            const double r = warp_sum16(acc);
            const int kk = lane % 5, kind = lane / 5, k = k0 + kk;
            if (lane < 15 && k <= n) {
                const size_t pk = (size_t)col * PK + k + (size_t)n * (n + 1) / 2;
                if (kind == 0) a.Hp[pk] = r * pscale;
                else if (kind == 1) a.Sp[pk] = r;
                else {
                    h[k] = r;                // the coefficients of the unscaled P
                    if constexpr (kAdj) hess[(size_t)n * a.nu_max + k] = r * pscale;
                }
            }
            if (k0 == 0) hh = __shfl_sync(0xffffffffu, r, 15);
        }
        if (n == nu - 1) break;
        __syncwarp();
        const bool from_overlap = a.reorth != 0;
        if (from_overlap) second_pass_from_overlap<32>(a.Sp + (size_t)col * PK, h, n, lane, 0xffffffffu);
        // sweep B: w = hu - U h (first pass) and the second-pass coefficients SU^T w,
        // sixteen k at a time (the first sixteen in the same sweep as the update); with the
        // second pass from S', sweep C alone subtracts both passes
        for (int k0 = 0; k0 <= (from_overlap ? -1 : n); k0 += 16) {
            double acc2[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc2[q] = 0.0;
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * 32 + lane;
                double2 w0, w1;
                ld4(P + 4 * p, w0, w1);
                if (k0 == 0) {
                    sub_basis(Uw, NP, p, h, n, w0, w1, sl + 1 < NS ? p + NP / NS : -1);
                    st4(P + 4 * p, w0, w1);
                }
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    if (k0 + kk <= n) {
                        double2 v0, v1;
                        if (sl + 1 < NS) prefetch_l2(SUw + (size_t)(k0 + kk) * vs + 4 * (p + 32));
                        ld4(SUw + (size_t)(k0 + kk) * vs + 4 * p, v0, v1);
                        acc2[kk] = fma4(v0, v1, w0, w1, acc2[kk]);
                    }
                }
            }
            const double r2 = warp_sum16(acc2);
            // the first-pass coefficients were last read by the update of the first
            // chunk, so the second-pass ones replace them in place
            __syncwarp();
            if (lane < 16 && k0 + lane <= n) h[k0 + lane] = r2;
            __syncwarp();
        }
        // sweep C: w -= U h (second pass)
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * 32 + lane;
            double2 w0, w1;
            ld4(P + 4 * p, w0, w1);
            sub_basis(Uw, NP, p, h, n, w0, w1, sl + 1 < NS ? p + NP / NS : -1);
            st4(P + 4 * p, w0, w1);
        }
        __syncwarp();
        // H w -> Q and S w -> the next SU slot in one pass, then beta
        double* SUn1 = SUw + (size_t)(n + 1) * vs;
        spmv_hs_w<32>(a.H, a.S, a.skr, ell, kmax, NS, P, Q, SUn1, lane, onsite, eself);
        double part = 0.0;
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * 32 + lane;
            double2 w0, w1, v0, v1;
            ld4(P + 4 * p, w0, w1);
            ld4(SUn1 + 4 * p, v0, v1);
            part = fma4(w0, w1, v0, v1, part);
        }
        const double beta2 = warp_sum(part);
        if (!(beta2 == beta2)) {   // NaN
            if (lane == 0) flag(a.status, DEV_NONFINITE);
            nu_eff = n + 1;
            break;
        }
        if (beta2 < -(a.breakdown_tol * a.breakdown_tol) * hh) {   // w^T S w < 0: S is not SPD
            if (lane == 0) flag(a.status, DEV_NOT_SPD);
            nu_eff = n + 1;
            break;
        }
        const double beta = sqrt(fmax(beta2, 0.0));
        if (beta <= a.breakdown_tol * sqrt(hh)) {
            nu_eff = n + 1;
            break;
        }
        if constexpr (kAdj) {
            if (lane == 0) hess[(size_t)n * a.nu_max + n + 1] = beta * pscale;
        }
        // u_{n+1} = w / beta, S u_{n+1} = S w / beta; H w stays in Q unscaled, with
        // H u_{n+1} = (H w) / beta by linearity (the next step's pscale). w here is the true
        // residual divided by the previous pscale (it was formed from the unscaled P), which
        // the normalisation cancels: beta, the breakdown and S-norm tests and u_{n+1} all take
        // the same factor or none.
        const double inv = 1.0 / beta;
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * 32 + lane;
            double2 w0, w1, v0, v1;
            ld4(P + 4 * p, w0, w1);
            ld4(SUn1 + 4 * p, v0, v1);
            w0.x *= inv; w0.y *= inv; w1.x *= inv; w1.y *= inv;
            v0.x *= inv; v0.y *= inv; v1.x *= inv; v1.y *= inv;
            st4(Uw + (size_t)(n + 1) * vs + 4 * p, w0, w1);
            st4(SUn1 + 4 * p, v0, v1);
        }
        pscale = inv;
        double* t = P;
        P = Q;
        Q = t;
        __syncwarp();
    }
    return nu_eff;
}


// ------------------------------------------------------------------------------------------------
// The same building blocks for a group of W lanes per column (W = 16: two columns per warp, one
// per half-warp; used by k_krylov_half). Shuffles and barriers take the group's own mask, so the
// two halves of a warp are independent. Kept apart from the one-warp forms above so that those
// compile exactly as before.
// The lanes of the calling thread's group of W lanes (the warp, or its half).
template <int W>
__device__ __forceinline__ unsigned group_mask() {
    return W == 32 ? 0xffffffffu : (0xffffu << (threadIdx.x & 16));
}

// Sum of 16 values held by every lane over the group (recursive halving on lane bits 3..0; for
// W = 32 then one exchange across bit 4): lane l of the group ends with the sum of value l & 15.
template <int W>
__device__ __forceinline__ double warp_sum16_w(double (&v)[16]) {
    const int lane = threadIdx.x & 31;
    const unsigned m = group_mask<W>();
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            double send = upper ? v[i] : v[i + w];
            double keep = upper ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(m, send, w);
        }
    }
    if (W == 32) return v[0] + __shfl_xor_sync(m, v[0], 16);
    return v[0];
}

// Sum of one value over the group.
template <int W>
__device__ __forceinline__ double group_sum(double v) {
    const unsigned m = group_mask<W>();
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
}

// y = A x on the cluster (lane-owned rows; x gathered from shared memory, y in shared or global
// memory). Each lane walks one list holding the entries of all its rows in slot order
// (entry.p4 low 16 bits: neighbour offset in x; high bits: the row's slot; `lane` is the lane
// within the group of W, `ent` the [kmax][W] lists), so lanes stop after
// their own entry count instead of after the widest row of every slot. Rows start from the
// on-site term: the diagonal of the on-site block of `dvals` (block index eself[p]), the
// identity when dvals is null, or zero when the on-site block is a list entry. With `skr` the
// off-site blocks are applied in their two-centre form (13 FP64 instructions instead of 16;
// which = 0 selects the H integrals, 1 the S integrals).
template <int W>
__device__ __forceinline__ void spmv_w(const double* __restrict__ vals, const double* __restrict__ skr,
                                     int which, const Ent* __restrict__ ent, int kmax, int NS,
                                     const double* x, double* y, int lane, bool onsite,
                                     const double* __restrict__ dvals, const int* eself) {
    for (int s = 0; s < NS; ++s) {
        const int p = s * W + lane, po = 4 * p;
        double2 o01 = make_double2(0.0, 0.0), o23 = make_double2(0.0, 0.0);
        if (onsite) {
            o01 = *reinterpret_cast<const double2*>(x + po);
            o23 = *reinterpret_cast<const double2*>(x + po + 2);
            const int es = eself[p];
            if (dvals && es >= 0) {
                const double* d = dvals + 16 * (size_t)es;
                o01.x *= __ldg(d); o01.y *= __ldg(d + 5); o23.x *= __ldg(d + 10); o23.y *= __ldg(d + 15);
            }
        }
        *reinterpret_cast<double2*>(y + po) = o01;
        *reinterpret_cast<double2*>(y + po + 2) = o23;
    }
    int cur = -1;
    double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
    for (int k = 0; k < kmax; ++k) {
        const Ent en = ent[W * k + lane];
        if (en.blk >= 0) {
            const int s = en.p4 >> 16, p4 = en.p4 & 0xffff;
            if (s != cur) {
                if (cur >= 0) {
                    double2* yo = reinterpret_cast<double2*>(y + 4 * (cur * W + lane));
                    yo[0] = make_double2(y0, y1);
                    yo[1] = make_double2(y2, y3);
                }
                cur = s;
                const double2* yi = reinterpret_cast<const double2*>(y + 4 * (s * W + lane));
                const double2 i01 = yi[0], i23 = yi[1];
                y0 = i01.x; y1 = i01.y; y2 = i23.x; y3 = i23.y;
            }
            const double2 x01 = *reinterpret_cast<const double2*>(x + p4);
            const double2 x23 = *reinterpret_cast<const double2*>(x + p4 + 2);
            if (skr) {
                // two-centre block: t = u.x_p; y_s += V_ss x_s + V_sp t;
                // y_p += V_pi x_p + (dV t - V_sp x_s) u,  dV = V_pp_sigma - V_pp_pi
                const double2* q = reinterpret_cast<const double2*>(skr + 12 * (size_t)en.blk);
                const double2 u01 = __ldg(q), u2_ = __ldg(q + 1);
                const double2 v01 = __ldg(q + 2 + 2 * which), v23 = __ldg(q + 3 + 2 * which);
                const double t = fma(u2_.x, x23.y, fma(u01.y, x23.x, u01.x * x01.y));
                y0 = fma(v01.y, t, fma(v01.x, x01.x, y0));
                const double aa = fma(v23.y, t, -v01.y * x01.x);
                y1 = fma(aa, u01.x, fma(v23.x, x01.y, y1));
                y2 = fma(aa, u01.y, fma(v23.x, x23.x, y2));
                y3 = fma(aa, u2_.x, fma(v23.x, x23.y, y3));
            } else {
                const double2* b2 = reinterpret_cast<const double2*>(vals + 16 * (size_t)en.blk);
                const double2 a0 = __ldg(b2 + 0), a1 = __ldg(b2 + 1), a2 = __ldg(b2 + 2), a3 = __ldg(b2 + 3);
                const double2 a4 = __ldg(b2 + 4), a5 = __ldg(b2 + 5), a6 = __ldg(b2 + 6), a7 = __ldg(b2 + 7);
                y0 = fma(a0.x, x01.x, fma(a0.y, x01.y, fma(a1.x, x23.x, fma(a1.y, x23.y, y0))));
                y1 = fma(a2.x, x01.x, fma(a2.y, x01.y, fma(a3.x, x23.x, fma(a3.y, x23.y, y1))));
                y2 = fma(a4.x, x01.x, fma(a4.y, x01.y, fma(a5.x, x23.x, fma(a5.y, x23.y, y2))));
                y3 = fma(a6.x, x01.x, fma(a6.y, x01.y, fma(a7.x, x23.x, fma(a7.y, x23.y, y3))));
            }
        }
    }
    if (cur >= 0) {
        double2* yo = reinterpret_cast<double2*>(y + 4 * (cur * W + lane));
        yo[0] = make_double2(y0, y1);
        yo[1] = make_double2(y2, y3);
    }
}

// Builds the view of atom J's cluster (every thread of the CTA, T threads, calls it) for slots of
// W lanes. Returns false, the same on every thread, when the cluster exceeds NA atoms or the
// lists exceed their capacity.
template <int W, int T>
__device__ __forceinline__ bool cluster_view_w(const KrylovArgs& a, int J, int NA, ClusterView& v) {
    __shared__ int sh_bad, sh_kmax, sh_nent;
    const int tid = threadIdx.x;
    const bool onsite = a.onsite_diag != 0;
    Ent* ell = v.ell;
    int* cl = v.cl;
    int* deg = v.deg;
    int* pos_of = v.pos_of;
    int* atom_at = v.atom_at;
    int* eoff = v.eoff;
    int* eself = v.eself;
    int n_at, cbase = 0;
    if (a.cl_ptr) { cbase = a.cl_ptr[J]; n_at = a.cl_ptr[J + 1] - cbase; }
    else n_at = a.n_atoms;
    if (n_at > NA) return false;   // uniform across the CTA
    for (int q = tid; q < n_at; q += T) cl[q] = a.cl_ptr ? a.cl_idx[cbase + q] : q;
    __syncthreads();
    for (int q = tid; q < n_at; q += T) {
        const int A = cl[q];
        int cnt = 0;
        for (int e = a.row_ptr[A]; e < a.row_ptr[A + 1]; ++e) {
            const int ce = a.col_idx[e];
            cnt += (!onsite || ce != A) && bsearch_sorted(cl, n_at, ce) >= 0;
        }
        deg[q] = cnt;
    }
    __syncthreads();
    const int NS = (n_at + W - 1) / W;
    balanced_positions<W, T>(n_at, NS, deg, pos_of, atom_at);
    // per-lane lists: the entries of the lane's rows in slot order
    if (tid < W) {
        const unsigned m = W == 32 ? 0xffffffffu : 0xffffu;
        int off = 0;
        for (int sl = 0; sl < NS; ++sl) {
            const int pp = sl * W + tid;
            const int q = atom_at[pp];
            eoff[pp] = off;
            off += q >= 0 ? deg[q] : 0;
        }
        int kmax = off, ntot = off;
        for (int o = W / 2; o > 0; o >>= 1) {
            kmax = max(kmax, __shfl_xor_sync(m, kmax, o));
            ntot += __shfl_xor_sync(m, ntot, o);
        }
        if (tid == 0) {
            sh_nent = ntot;
            sh_kmax = kmax;
            sh_bad = kmax * W > NA * a.deg_max;
        }
    }
    __syncthreads();
    if (sh_bad) return false;
    const int kmax = sh_kmax;
    for (int q = tid; q < kmax * W; q += T) ell[q] = Ent{0, -1};
    __syncthreads();
    for (int p = tid; p < NS * W; p += T) {
        const int q = atom_at[p];
        const int sl = p / W, l = p % W;
        int k = eoff[p];
        int es = -1;
        if (q >= 0) {
            const int A = cl[q];
            for (int e = a.row_ptr[A]; e < a.row_ptr[A + 1]; ++e) {
                const int ce = a.col_idx[e];
                if (onsite && ce == A) {
                    es = e;
                    continue;
                }
                const int b = bsearch_sorted(cl, n_at, ce);
                if (b >= 0) ell[W * (k++) + l] = Ent{(4 * pos_of[b]) | (sl << 16), e};
            }
        }
        eself[p] = es;
    }
    __syncthreads();
    v.n_at = n_at;
    v.NS = NS;
    v.kmax = kmax;
    v.nent = sh_nent;
    return true;
}

// Forward Krylov recursion of column j = 4 J + alpha by one warp (the reading of the module
// header of krylov.cu): leaves U and SU in Uw, SUw ([k][position][orbital]) and writes H', S'
// (packed upper) and row j of U, SU, HU of the column. With kAdj it also keeps HU in HUw and the
// Gram-Schmidt coefficients in hess[n][k] (row stride nu_max): SU_k . HU_n for k <= n (the
// first pass) and beta_n at k = n + 1, which the adjoint needs. A and B are the warp's two
// shared vectors (u_1, then by turns H u_n -> w and the products H w of the next vector), h its
// coefficient buffer. The H and S products of each new vector are formed together from w
// (spmv_hs_w); the S product is scaled by 1 / beta with w, the H product is kept unscaled and its
// scale carried as a scalar (pscale). Returns nu_eff (nu_out: the column's nu), or 0
// for bad input (flagged).
template <bool kAdj, int W>
__device__ __forceinline__ int column_forward_w(const KrylovArgs& a, const ClusterView& v, int J, int alpha,
                                              double* A, double* B, double* h, double* Uw, double* SUw,
                                              double* HUw, double* hess, int& nu_out, int& jp_out) {
    const int lane = threadIdx.x & (W - 1);      // lane within the column's group
    const unsigned gm = group_mask<W>();
    const bool onsite = a.onsite_diag != 0;
    const int n_at = v.n_at, NS = v.NS, kmax = v.kmax;
    const int* cl = v.cl;
    const int* pos_of = v.pos_of;
    const Ent* ell = v.ell;
    const int* eself = v.eself;
    const int PK = a.nu_max * (a.nu_max + 1) / 2;
    const int j = 4 * J + alpha;
    const int col = j - 4 * a.atom_begin;
    const int NP = NS * W;
    const int nu = min(nu_for(a, n_at), a.nu_max);
    nu_out = nu;
    const int aJ = bsearch_sorted(cl, n_at, J);
    int eJJ = -1;
    for (int e = a.row_ptr[J]; e < a.row_ptr[J + 1]; ++e)
        if (a.col_idx[e] == J) eJJ = e;
    const double sjj = eJJ >= 0 ? a.S[16 * (size_t)eJJ + 5 * alpha] : -1.0;
    if (aJ < 0 || !(sjj > 0.0)) {   // no diagonal block or S_jj <= 0: bad input
        if (lane == 0) { flag(a.status, DEV_ARG); a.nu_eff[j] = 0; }
        return 0;
    }
    const int jp = 4 * pos_of[aJ] + alpha;
    jp_out = jp;
    const size_t vs = (size_t)NP * 4;                    // one basis vector

    for (int q = lane; q < NP * 4; q += W) A[q] = 0.0;
    __syncwarp(gm);
    if (lane == 0) A[jp] = 1.0 / sqrt(sjj);
    __syncwarp(gm);
    // H u_1 -> B, S u_1 -> SU[0]; u_1 -> U[0]
    spmv_hs_w<W>(a.H, a.S, a.skr, ell, kmax, NS, A, B, SUw, lane, onsite, eself);
    for (int sl = 0; sl < NS; ++sl) {
        const int p = sl * W + lane;
        double2 x0, x1;
        ld4(A + 4 * p, x0, x1);
        st4(Uw + 4 * (size_t)p, x0, x1);
    }
    __syncwarp(gm);

    // P holds H u_n at the top of step n (then w); the products of the next basis vector go to Q
    double* P = B;
    double* Q = A;
    // H u_n = pscale P: the H product of each new vector stays unscaled in P, and the values
    // formed from it (H', the first-pass coefficients) are scaled once as scalars
    double pscale = 1.0;
    int nu_eff = nu;
    for (int n = 0; n < nu; ++n) {
        double* SUn = SUw + (size_t)n * vs;
        if constexpr (kAdj) {
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * W + lane;
                double2 x0, x1;
                ld4(P + 4 * p, x0, x1);
                x0.x *= pscale; x0.y *= pscale; x1.x *= pscale; x1.y *= pscale;
                st4(HUw + (size_t)n * vs + 4 * p, x0, x1);
            }
        }
        if (lane == 0) {
            a.urow[(size_t)col * a.nu_max + n] = Uw[(size_t)n * vs + jp];
            a.surow[(size_t)col * a.nu_max + n] = SUn[jp];
            a.hurow[(size_t)col * a.nu_max + n] = P[jp] * pscale;
        }
        // pass A: H'[k][n], S'[k][n] and the first CGS coefficients, k <= n, five k at a time
        double hh = 0.0;
        for (int k0 = 0; k0 <= n; k0 += 5) {
            double acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.0;
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * W + lane;
                // the rows this chunk reads next: the next position, else the next chunk's first
                const int pn = sl + 1 < NS ? p + W : lane;
                const int kn = sl + 1 < NS ? k0 : k0 + 5;
                double2 hu0, hu1, su0, su1;
                ld4(P + 4 * p, hu0, hu1);
                ld4(SUn + 4 * p, su0, su1);
                if (k0 == 0) acc[15] = fma4(hu0, hu1, hu0, hu1, acc[15]);
#pragma unroll
                for (int kk = 0; kk < 5; ++kk) {
                    const int k = k0 + kk;
                    if (kn + kk <= n) {
                        prefetch_l2(Uw + (size_t)(kn + kk) * vs + 4 * pn);
                        prefetch_l2(SUw + (size_t)(kn + kk) * vs + 4 * pn);
                    }
                    if (k <= n) {
                        double2 u0, u1, v0, v1;
                        ld4(Uw + (size_t)k * vs + 4 * p, u0, u1);
                        ld4(SUw + (size_t)k * vs + 4 * p, v0, v1);
                        acc[kk] = fma4(u0, u1, hu0, hu1, acc[kk]);
                        acc[5 + kk] = fma4(u0, u1, su0, su1, acc[5 + kk]);
                        acc[10 + kk] = fma4(v0, v1, hu0, hu1, acc[10 + kk]);
                    }
                }
            }
            const double r = warp_sum16_w<W>(acc);
            const int kk = lane % 5, kind = lane / 5, k = k0 + kk;
            if (lane < 15 && k <= n) {
                const size_t pk = (size_t)col * PK + k + (size_t)n * (n + 1) / 2;
                if (kind == 0) a.Hp[pk] = r * pscale;
                else if (kind == 1) a.Sp[pk] = r;
                else {
                    h[k] = r;                // the coefficients of the unscaled P
                    if constexpr (kAdj) hess[(size_t)n * a.nu_max + k] = r * pscale;
                }
            }
            if (k0 == 0) hh = __shfl_sync(gm, r, ((threadIdx.x & 31) & ~(W - 1)) + 15);
        }
        if (n == nu - 1) break;
        __syncwarp(gm);
        const bool from_overlap = a.reorth != 0;
        if (from_overlap) second_pass_from_overlap<W>(a.Sp + (size_t)col * PK, h, n, lane, gm);
        // sweep B: w = hu - U h (first pass) and the second-pass coefficients SU^T w,
        // sixteen k at a time (the first sixteen in the same sweep as the update); with the
        // second pass from S', sweep C alone subtracts both passes
        for (int k0 = 0; k0 <= (from_overlap ? -1 : n); k0 += 16) {
            double acc2[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc2[q] = 0.0;
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * W + lane;
                double2 w0, w1;
                ld4(P + 4 * p, w0, w1);
                if (k0 == 0) {
                    sub_basis(Uw, NP, p, h, n, w0, w1, sl + 1 < NS ? p + W : -1);
                    st4(P + 4 * p, w0, w1);
                }
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    if (k0 + kk <= n) {
                        double2 v0, v1;
                        if (sl + 1 < NS) prefetch_l2(SUw + (size_t)(k0 + kk) * vs + 4 * (p + W));
                        ld4(SUw + (size_t)(k0 + kk) * vs + 4 * p, v0, v1);
                        acc2[kk] = fma4(v0, v1, w0, w1, acc2[kk]);
                    }
                }
            }
            const double r2 = warp_sum16_w<W>(acc2);
            // the first-pass coefficients were last read by the update of the first
            // chunk, so the second-pass ones replace them in place
            __syncwarp(gm);
            if (lane < 16 && k0 + lane <= n) h[k0 + lane] = r2;
            __syncwarp(gm);
        }
        // sweep C: w -= U h (second pass)
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * W + lane;
            double2 w0, w1;
            ld4(P + 4 * p, w0, w1);
            sub_basis(Uw, NP, p, h, n, w0, w1, sl + 1 < NS ? p + W : -1);
            st4(P + 4 * p, w0, w1);
        }
        __syncwarp(gm);
        // H w -> Q and S w -> the next SU slot in one pass, then beta
        double* SUn1 = SUw + (size_t)(n + 1) * vs;
        spmv_hs_w<W>(a.H, a.S, a.skr, ell, kmax, NS, P, Q, SUn1, lane, onsite, eself);
        double part = 0.0;
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * W + lane;
            double2 w0, w1, v0, v1;
            ld4(P + 4 * p, w0, w1);
            ld4(SUn1 + 4 * p, v0, v1);
            part = fma4(w0, w1, v0, v1, part);
        }
        const double beta2 = group_sum<W>(part);
        if (!(beta2 == beta2)) {   // NaN
            if (lane == 0) flag(a.status, DEV_NONFINITE);
            nu_eff = n + 1;
            break;
        }
        if (beta2 < -(a.breakdown_tol * a.breakdown_tol) * hh) {   // w^T S w < 0: S is not SPD
            if (lane == 0) flag(a.status, DEV_NOT_SPD);
            nu_eff = n + 1;
            break;
        }
        const double beta = sqrt(fmax(beta2, 0.0));
        if (beta <= a.breakdown_tol * sqrt(hh)) {
            nu_eff = n + 1;
            break;
        }
        if constexpr (kAdj) {
            if (lane == 0) hess[(size_t)n * a.nu_max + n + 1] = beta * pscale;
        }
        // u_{n+1} = w / beta, S u_{n+1} = S w / beta; H w stays in Q unscaled, with
        // H u_{n+1} = (H w) / beta by linearity (the next step's pscale). w here is the true
        // residual divided by the previous pscale (it was formed from the unscaled P), which
        // the normalisation cancels: beta, the breakdown and S-norm tests and u_{n+1} all take
        // the same factor or none.
        const double inv = 1.0 / beta;
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * W + lane;
            double2 w0, w1, v0, v1;
            ld4(P + 4 * p, w0, w1);
            ld4(SUn1 + 4 * p, v0, v1);
            w0.x *= inv; w0.y *= inv; w1.x *= inv; w1.y *= inv;
            v0.x *= inv; v0.y *= inv; v1.x *= inv; v1.y *= inv;
            st4(Uw + (size_t)(n + 1) * vs + 4 * p, w0, w1);
            st4(SUn1 + 4 * p, v0, v1);
        }
        pscale = inv;
        double* t = P;
        P = Q;
        Q = t;
        __syncwarp(gm);
    }
    return nu_eff;
}

}  // namespace elses
