// a3 + a4: per-column Krylov build in the S inner product and the projection H' = U^T H U,
// S' = U^T S U, for every column j = 4J + alpha of a batch of atoms.
//
// The paper generates G = (zS - H)^-1 column by column (Eq. 1 with b = e_j) with a Krylov
// solver (the paper's multiple Arnoldi method) on the local cluster of j. The reading built
// here (the oracle's):
//     u_1 = e_j / sqrt(S_jj); for n = 1..nu: HU_n = H_C u_n; stop at n = nu;
//     w = HU_n; two classical Gram-Schmidt passes h = SU^T w, w -= U h;
//     Sw = S_C w; beta = sqrt(w^T Sw); stop if beta <= tol ||HU_n||_2; u_{n+1} = w / beta,
// with SU_{n+1} = Sw / beta and HU_{n+1} = Hw / beta (the products of u_{n+1} by linearity,
// Hw and Sw formed in one pass over the cluster; the oracle forms S u_{n+1} and H u_{n+1} by
// products, which agree to rounding). H'[k][n] = u_k . HU_n and S'[k][n] = u_k . SU_n are formed
// for k <= n as the columns appear (the oracle symmetrises full products; same values to
// rounding). With KrylovArgs::reorth = 1 the second pass takes its coefficients from S'
// instead of a second product with SU (second_pass_from_overlap, krylov.cuh) and one sweep of
// the basis subtracts both passes: the same space to rounding, with a third fewer basis reads
// and dense flops.
//
// GB300 layout: one CTA of 4 warps per atom J, one warp per orbital column alpha; the CTA
// builds an ELL view of the cluster sub-matrix (atoms sorted by in-cluster degree and assigned
// to lanes so that their list lengths balance) in shared memory once for the 4
// columns. Each lane owns whole atoms (4 rows); the sparse products gather the source vector
// from shared memory and stream the 4x4 FP64 blocks (the 4 warps of a CTA read the same blocks,
// which L1 serves). The S-inner products of CGS2 and the projection are per-lane partial sums
// reduced by recursive halving (one addition per value). The bases U and SU stay in per-CTA
// global scratch in [k][position][orbital] order (coalesced 32-byte rows per lane). FP64
// everywhere; no tensor cores (the work is sparse and FP64).
#include <algorithm>

#include "krylov.cuh"

namespace elses {

size_t krylov_smem_bytes(int na_max, int deg_max) {
    size_t b = 0;
    b += sizeof(double) * (size_t)kWarpsPerAtom * 2 * na_max * 4;   // u and hu / w per warp
    b += sizeof(double) * (size_t)kWarpsPerAtom * kMaxNu;            // CGS coefficients
    b += view_bytes(na_max, deg_max);                                // ELL and lists
    return (b + 15) & ~(size_t)15;
}

// kStore: the bases of every column are kept in a.bstore (with HU, the Gram-Schmidt
// coefficients and H') for the exact-gradient kernel, instead of the per-CTA scratch.
// kMinB: resident CTAs per SM the register budget is set for -- 3 (168 registers), or 4 (128
// registers, a few hundred bytes of spills to L1-cached local memory) for size classes whose
// shared memory leaves room for a fourth CTA; the autotuner times both.
template <bool kStore, int kMinB>
__global__ void __launch_bounds__(kThreads, kMinB) k_krylov(const KrylovArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NA = a.na_max;
    double* vec = reinterpret_cast<double*>(smem_raw);
    double* hbuf = vec + (size_t)kWarpsPerAtom * 2 * NA * 4;
    ClusterView v;
    carve_view(reinterpret_cast<unsigned char*>(hbuf + kWarpsPerAtom * kMaxNu), NA, a.deg_max, v);
    __shared__ int sh_atom;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t warp_scratch = (size_t)2 * a.nu_max * NA * 4;
    double* Uw = a.scratch + (size_t)blockIdx.x * kWarpsPerAtom * warp_scratch + (size_t)warp * warp_scratch;
    double* SUw = Uw + (size_t)a.nu_max * NA * 4;
    const int n_batch = a.n_items;

    for (int iter = 0;; ++iter) {
        if (tid == 0) {
            const int idx = a.queue ? atomicAdd(a.queue, 1) : blockIdx.x + iter * gridDim.x;
            int atom = -1;
            if (idx < n_batch) atom = a.order[idx];
            sh_atom = atom;
        }
        __syncthreads();
        const int J = sh_atom;
        if (J < 0) break;
        if (!cluster_view(a, J, NA, v)) {
            if (tid == 0) flag(a.status, DEV_CAPACITY);
            __syncthreads();
            continue;
        }

        // ---------------------------------------------------------------- column alpha = warp
        do {
            const int alpha = warp;
            const int j = 4 * J + alpha;
            const int n_at = v.n_at, NP = v.NS * 32;
            double* A = vec + (size_t)(warp * 2) * NA * 4;    // the warp's two shared vectors:
            double* B = A + (size_t)NA * 4;                      // H u_n then w, and H w
            int nu = 0, jp = 0;
            double *Ucol = Uw, *SUcol = SUw, *HUcol = nullptr, *hess = nullptr;
            if constexpr (kStore) {
                Ucol = a.bstore + (size_t)j * a.bstride;
                SUcol = Ucol + a.bvec;
                HUcol = SUcol + a.bvec;
                hess = HUcol + a.bvec;
            }
            const int nu_eff = column_forward<kStore>(a, v, J, alpha, A, B, hbuf + warp * kMaxNu, Ucol, SUcol,
                                                      HUcol, hess, nu, jp);
            if (nu_eff <= 0) break;   // bad input (flagged); the CTA barrier follows
            if constexpr (kStore) {   // H' of the column beside its bases
                __syncwarp();
                const int PK = a.nu_max * (a.nu_max + 1) / 2;
                const double* hp = a.Hp + (size_t)(j - 4 * a.atom_begin) * PK;
                double* out = hess + (size_t)a.nu_max * a.nu_max;
                for (int q = lane; q < PK; q += 32) out[q] = hp[q];
            }
            if (lane == 0) {
                a.nu_eff[j] = nu_eff;
                if (nu_eff < nu) flag(a.status, DEV_BREAKDOWN);
                if (a.flops) atomicAdd(a.flops, column_flops(a, n_at, v.nent, nu_eff, a.reorth != 0));
            }
            __syncwarp();
            // pattern rows of U for rho / G: blocks e = (J, I) of row J, orbital r of atom I
            if (a.UP) {
                const int e0 = a.row_ptr[J], ne = a.row_ptr[J + 1] - e0;
                for (int q = lane; q < ne * 4; q += 32) {
                    const int e = e0 + (q >> 2), r = q & 3;
                    const int b = bsearch_sorted(v.cl, n_at, a.col_idx[e]);
                    const int p = v.pos_of[b];
                    double* out = a.UP + ((size_t)((e - a.up_block0) * 4 + alpha) * 4 + r) * a.nu_max;
                    for (int k = 0; k < nu_eff; ++k) out[k] = Ucol[4 * ((size_t)k * NP + p) + r];
                }
            }
        } while (0);
        __syncthreads();
    }
}

// The same recursion with two columns per warp, one per half-warp (W = 16; the module header of
// krylov.cuh): a CTA of 2 warps per atom J, column alpha = threadIdx.x / 16, for clusters whose
// last slot of 32 atoms would be at most half full (na_max a multiple of 16). Without kept bases.
constexpr int kHalfThreads = 16 * kWarpsPerAtom;
__global__ void __launch_bounds__(kHalfThreads, 6) k_krylov_half(const KrylovArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NA = a.na_max;
    double* vec = reinterpret_cast<double*>(smem_raw);
    double* hbuf = vec + (size_t)kWarpsPerAtom * 2 * NA * 4;
    ClusterView v;
    carve_view(reinterpret_cast<unsigned char*>(hbuf + kWarpsPerAtom * kMaxNu), NA, a.deg_max, v);
    __shared__ int sh_atom;

    const int tid = threadIdx.x, lane = tid & 15, alpha = tid >> 4;
    const unsigned gm = group_mask<16>();
    const size_t col_scratch = (size_t)2 * a.nu_max * NA * 4;
    double* Uw = a.scratch + (size_t)blockIdx.x * kWarpsPerAtom * col_scratch + (size_t)alpha * col_scratch;
    double* SUw = Uw + (size_t)a.nu_max * NA * 4;
    const int n_batch = a.n_items;

    for (int iter = 0;; ++iter) {
        if (tid == 0) {
            const int idx = a.queue ? atomicAdd(a.queue, 1) : blockIdx.x + iter * gridDim.x;
            int atom = -1;
            if (idx < n_batch) atom = a.order[idx];
            sh_atom = atom;
        }
        __syncthreads();
        const int J = sh_atom;
        if (J < 0) break;
        if (!cluster_view_w<16, kHalfThreads>(a, J, NA, v)) {
            if (tid == 0) flag(a.status, DEV_CAPACITY);
            __syncthreads();
            continue;
        }
        do {
            const int j = 4 * J + alpha;
            const int n_at = v.n_at, NP = v.NS * 16;
            double* A = vec + (size_t)(alpha * 2) * NA * 4;
            double* B = A + (size_t)NA * 4;
            int nu = 0, jp = 0;
            const int nu_eff = column_forward_w<false, 16>(a, v, J, alpha, A, B, hbuf + alpha * kMaxNu, Uw, SUw,
                                                         nullptr, nullptr, nu, jp);
            if (nu_eff <= 0) break;
            if (lane == 0) {
                a.nu_eff[j] = nu_eff;
                if (nu_eff < nu) flag(a.status, DEV_BREAKDOWN);
                if (a.flops) atomicAdd(a.flops, column_flops(a, n_at, v.nent, nu_eff, a.reorth != 0));
            }
            __syncwarp(gm);
            if (a.UP) {
                const int e0 = a.row_ptr[J], ne = a.row_ptr[J + 1] - e0;
                for (int q = lane; q < ne * 4; q += 16) {
                    const int e = e0 + (q >> 2), r = q & 3;
                    const int b = bsearch_sorted(v.cl, n_at, a.col_idx[e]);
                    const int p = v.pos_of[b];
                    double* out = a.UP + ((size_t)((e - a.up_block0) * 4 + alpha) * 4 + r) * a.nu_max;
                    for (int k = 0; k < nu_eff; ++k) out[k] = Uw[4 * ((size_t)k * NP + p) + r];
                }
            }
        } while (0);
        __syncthreads();
    }
}

int krylov_half_blocks_per_sm(int na_max, int deg_max) {
    const size_t smem = krylov_smem_bytes(na_max, deg_max);
    smem_at_least(k_krylov_half, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_krylov_half, kHalfThreads, smem);
    return nb;
}

int krylov_blocks_per_sm(int na_max, int deg_max) {
    const size_t smem = krylov_smem_bytes(na_max, deg_max);
    smem_at_least(k_krylov<false, 3>, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_krylov<false, 3>, kThreads, smem);
    return nb;
}

int krylov_blocks_per_sm_max(int na_max, int deg_max) {
    const size_t smem = krylov_smem_bytes(na_max, deg_max);
    smem_at_least(k_krylov<false, 4>, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_krylov<false, 4>, kThreads, smem);
    return std::max(nb, krylov_blocks_per_sm(na_max, deg_max));
}

void krylov_columns(const KrylovArgs& a, int grid, int ctas_per_sm, cudaStream_t st) {
    const size_t smem = krylov_smem_bytes(a.na_max, a.deg_max);
    if (a.half && !a.bstore) {
        smem_at_least(k_krylov_half, smem);
        k_krylov_half<<<grid, kHalfThreads, smem, st>>>(a);
    } else if (a.bstore) {
        smem_at_least(k_krylov<true, 3>, smem);
        k_krylov<true, 3><<<grid, kThreads, smem, st>>>(a);
    } else if (ctas_per_sm >= 4) {
        smem_at_least(k_krylov<false, 4>, smem);
        k_krylov<false, 4><<<grid, kThreads, smem, st>>>(a);
    } else {
        smem_at_least(k_krylov<false, 3>, smem);
        k_krylov<false, 3><<<grid, kThreads, smem, st>>>(a);
    }
}

}  // namespace elses
