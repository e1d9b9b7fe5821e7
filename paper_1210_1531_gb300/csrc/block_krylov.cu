// Block-start Krylov build per atom (the alternative reading of the multiple Arnoldi method):
// the 4 orbitals of atom J start one block Krylov space K(H_C, E_J), E_J = [e_4J .. e_4J+3],
// shared by the atom's 4 columns of Eq. 1. Its S-orthonormal basis is the band form of block
// Arnoldi (lag 4): the starting vectors S-orthonormalised, then u_{m+4} = CGS2(H u_m) against
// every basis vector so far, normalised in the S norm; the build stops extending at nu vectors or
// when beta <= tol ||H u_m||_2. H' = U^T H U and S' = U^T S U (upper triangles, as in the
// per-column kernel) are written for each of the 4 columns, with rows j of U, SU and HU and the
// pattern rows of U, so the eigensolver, bisection, density and forces run unchanged.
//
// GB300 form: one CTA of 4 warps per atom, the basis U, SU in per-CTA global scratch shared by
// the warps. A block step processes m = m0 .. m0+3 in parallel (warp alpha: H u_{m0+alpha}, its
// projection entries, CGS2 against the n_b vectors that existed when the step began, and S w),
// then the four candidates are finished in order (warp alpha: CGS2 against the new vectors of
// this step, with S w updated by linearity, the breakdown test and the normalisation), one warp
// at a time with the CTA barrier between. The same vectors as CGS2 against all vectors at once,
// to rounding.
#include "krylov.cuh"

namespace elses {

namespace {

// CGS2 of w (warp's shared vector B, lanes over rows) against basis vectors [k_lo, k_hi) of U /
// SU: h = SU^T w, w -= U h, twice. hb: the warp's coefficient buffer.
__device__ __forceinline__ void cgs2_range(const double* Ub, const double* SUb, int NS, size_t vs, int k_lo, int k_hi,
                                           double* B, double* hb, int lane) {
    for (int pass = 0; pass < 2; ++pass) {
        for (int k0 = k_lo; k0 < k_hi; k0 += 16) {
            double acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.0;
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * 32 + lane;
                double2 w0, w1;
                ld4(B + 4 * p, w0, w1);
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    if (k0 + kk < k_hi) {
                        double2 v0, v1;
                        ld4(SUb + (size_t)(k0 + kk) * vs + 4 * p, v0, v1);
                        acc[kk] = fma4(v0, v1, w0, w1, acc[kk]);
                    }
                }
            }
            const double r = warp_sum16(acc);
            __syncwarp();
            if (lane < 16 && k0 + lane < k_hi) hb[k0 + lane] = r;
            __syncwarp();
        }
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * 32 + lane;
            double2 w0, w1;
            ld4(B + 4 * p, w0, w1);
            for (int k = k_lo; k < k_hi; ++k) {
                double2 u0, u1;
                ld4(Ub + (size_t)k * vs + 4 * p, u0, u1);
                const double hk = hb[k];
                w0.x = fma(-u0.x, hk, w0.x); w0.y = fma(-u0.y, hk, w0.y);
                w1.x = fma(-u1.x, hk, w1.x); w1.y = fma(-u1.y, hk, w1.y);
            }
            st4(B + 4 * p, w0, w1);
        }
        __syncwarp();
    }
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 3) k_block_krylov(const KrylovArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NA = a.na_max, nm = a.nu_max;
    double* vec = reinterpret_cast<double*>(smem_raw);
    double* hbuf = vec + (size_t)kWarpsPerAtom * 2 * NA * 4;
    ClusterView v;
    carve_view(reinterpret_cast<unsigned char*>(hbuf + kWarpsPerAtom * kMaxNu), NA, a.deg_max, v);
    __shared__ int sh_atom, sh_nb, sh_ext, sh_nueff, sh_bad;
    __shared__ double sh_hh[kWarpsPerAtom];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool onsite = a.onsite_diag != 0;
    const size_t cta_scratch = (size_t)(2 * nm + kWarpsPerAtom) * NA * 4;
    double* Ub = a.scratch + (size_t)blockIdx.x * cta_scratch;
    double* SUb = Ub + (size_t)nm * NA * 4;
    double* Sw = SUb + (size_t)nm * NA * 4 + (size_t)warp * NA * 4;   // this warp's S w
    double* A = vec + (size_t)(warp * 2) * NA * 4;
    double* B = A + (size_t)NA * 4;
    double* hb = hbuf + warp * kMaxNu;
    const int PK = nm * (nm + 1) / 2;

    for (int iter = 0;; ++iter) {
        if (tid == 0) {
            const int idx = a.queue ? atomicAdd(a.queue, 1) : blockIdx.x + iter * gridDim.x;
            sh_atom = idx < a.n_items ? a.order[idx] : -1;
        }
        __syncthreads();
        const int J = sh_atom;
        if (J < 0) break;
        if (!cluster_view(a, J, NA, v)) {
            if (tid == 0) flag(a.status, DEV_CAPACITY);
            __syncthreads();
            continue;
        }
        const int n_at = v.n_at, NS = v.NS, NP = NS * 32;
        const size_t vs = (size_t)NP * 4;
        const int nu = min(nu_for(a, n_at), nm);
        const int aJ = bsearch_sorted(v.cl, n_at, J);
        const int col0 = 4 * J - 4 * a.atom_begin;          // batch-local column of alpha = 0
        const int jp0 = aJ >= 0 ? 4 * v.pos_of[aJ] : 0;      // row of e_4J in the cluster vectors
        if (tid == 0) { sh_nb = 0; sh_ext = 1; sh_nueff = nu; sh_bad = aJ < 0; }
        __syncthreads();

        // ---------------------------------------------------------------- starting vectors
        for (int s = 0; s < kWarpsPerAtom && !sh_bad; ++s) {
            if (warp == s) {
                for (int q = lane; q < NP * 4; q += 32) B[q] = 0.0;
                __syncwarp();
                if (lane == 0) B[jp0 + s] = 1.0;
                __syncwarp();
                cgs2_range(Ub, SUb, NS, vs, 0, s, B, hb, lane);
                spmv(a.S, a.skr, 1, v.ell, v.kmax, NS, B, Sw, lane, onsite, nullptr, v.eself);
                double part = 0.0;
                for (int sl = 0; sl < NS; ++sl) {
                    const int p = sl * 32 + lane;
                    double2 w0, w1, s0, s1;
                    ld4(B + 4 * p, w0, w1);
                    ld4(Sw + 4 * p, s0, s1);
                    part = fma4(w0, w1, s0, s1, part);
                }
                const double beta2 = warp_sum(part);
                if (!(beta2 > 0.0)) {   // NaN, or a start vector of S-norm <= 0: S is not SPD
                    if (lane == 0) { flag(a.status, beta2 == beta2 ? DEV_NOT_SPD : DEV_NONFINITE); sh_bad = 1; }
                } else {
                    const double inv = 1.0 / sqrt(beta2);
                    for (int sl = 0; sl < NS; ++sl) {
                        const int p = sl * 32 + lane;
                        double2 w0, w1, s0, s1;
                        ld4(B + 4 * p, w0, w1);
                        ld4(Sw + 4 * p, s0, s1);
                        w0.x *= inv; w0.y *= inv; w1.x *= inv; w1.y *= inv;
                        s0.x *= inv; s0.y *= inv; s1.x *= inv; s1.y *= inv;
                        st4(Ub + (size_t)s * vs + 4 * p, w0, w1);
                        st4(SUb + (size_t)s * vs + 4 * p, s0, s1);
                    }
                }
            }
            __syncthreads();
        }
        if (sh_bad) {
            if (tid < kWarpsPerAtom) a.nu_eff[4 * J + tid] = 0;
            __syncthreads();
            continue;
        }
        if (tid == 0) sh_nb = kWarpsPerAtom;
        __syncthreads();

        // ---------------------------------------------------------------- block steps
        for (int m0 = 0; m0 < sh_nueff; m0 += kWarpsPerAtom) {
            const int nb = sh_nb;                    // basis size when the step begins
            const int m = m0 + warp;
            const bool active = m < sh_nueff;
            const bool make = active && sh_ext && nb + warp < nu;
            if (active) {
                // H u_m
                for (int sl = 0; sl < NS; ++sl) {
                    const int p = sl * 32 + lane;
                    double2 x0, x1;
                    ld4(Ub + (size_t)m * vs + 4 * p, x0, x1);
                    st4(A + 4 * p, x0, x1);
                }
                __syncwarp();
                spmv(a.H, a.skr, 0, v.ell, v.kmax, NS, A, B, lane, onsite, a.H, v.eself);
                __syncwarp();
                if (lane < kWarpsPerAtom) {
                    const size_t o = (size_t)(col0 + lane) * nm + m;
                    a.urow[o] = Ub[(size_t)m * vs + jp0 + lane];
                    a.surow[o] = SUb[(size_t)m * vs + jp0 + lane];
                    a.hurow[o] = B[jp0 + lane];
                }
                // H'[k][m], S'[k][m] (k <= m) and the first CGS coefficients (k < nb)
                const double* SUm = SUb + (size_t)m * vs;
                double hh = 0.0;
                for (int k0 = 0; k0 < nb; k0 += 5) {
                    double acc[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
                    for (int sl = 0; sl < NS; ++sl) {
                        const int p = sl * 32 + lane;
                        double2 hu0, hu1, su0, su1;
                        ld4(B + 4 * p, hu0, hu1);
                        ld4(SUm + 4 * p, su0, su1);
                        if (k0 == 0) acc[15] = fma4(hu0, hu1, hu0, hu1, acc[15]);
#pragma unroll
                        for (int kk = 0; kk < 5; ++kk) {
                            const int k = k0 + kk;
                            if (k < nb) {
                                double2 u0, u1, v0, v1;
                                ld4(Ub + (size_t)k * vs + 4 * p, u0, u1);
                                ld4(SUb + (size_t)k * vs + 4 * p, v0, v1);
                                acc[kk] = fma4(u0, u1, hu0, hu1, acc[kk]);
                                acc[5 + kk] = fma4(u0, u1, su0, su1, acc[5 + kk]);
                                acc[10 + kk] = fma4(v0, v1, hu0, hu1, acc[10 + kk]);
                            }
                        }
                    }
                    const double r = warp_sum16(acc);
                    const int kk = lane % 5, kind = lane / 5, k = k0 + kk;
                    if (lane < 15 && k < nb) {
                        if (kind == 2) {
                            hb[k] = r;
                        } else if (k <= m) {
                            const size_t pk = k + (size_t)m * (m + 1) / 2;
                            double* P = kind == 0 ? a.Hp : a.Sp;
#pragma unroll
                            for (int c = 0; c < kWarpsPerAtom; ++c) P[(size_t)(col0 + c) * PK + pk] = r;
                        }
                    }
                    if (k0 == 0) hh = __shfl_sync(0xffffffffu, r, 15);
                }
                __syncwarp();
                if (make) {
                    // first pass with the coefficients above, then a second full pass
                    for (int sl = 0; sl < NS; ++sl) {
                        const int p = sl * 32 + lane;
                        double2 w0, w1;
                        ld4(B + 4 * p, w0, w1);
                        sub_basis(Ub, NP, p, hb, nb - 1, w0, w1);
                        st4(B + 4 * p, w0, w1);
                    }
                    __syncwarp();
                    for (int k0 = 0; k0 < nb; k0 += 16) {
                        double acc[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc[q] = 0.0;
                        for (int sl = 0; sl < NS; ++sl) {
                            const int p = sl * 32 + lane;
                            double2 w0, w1;
                            ld4(B + 4 * p, w0, w1);
#pragma unroll
                            for (int kk = 0; kk < 16; ++kk) {
                                if (k0 + kk < nb) {
                                    double2 v0, v1;
                                    ld4(SUb + (size_t)(k0 + kk) * vs + 4 * p, v0, v1);
                                    acc[kk] = fma4(v0, v1, w0, w1, acc[kk]);
                                }
                            }
                        }
                        const double r2 = warp_sum16(acc);
                        __syncwarp();
                        if (lane < 16 && k0 + lane < nb) hb[k0 + lane] = r2;
                        __syncwarp();
                    }
                    for (int sl = 0; sl < NS; ++sl) {
                        const int p = sl * 32 + lane;
                        double2 w0, w1;
                        ld4(B + 4 * p, w0, w1);
                        sub_basis(Ub, NP, p, hb, nb - 1, w0, w1);
                        st4(B + 4 * p, w0, w1);
                    }
                    __syncwarp();
                    spmv(a.S, a.skr, 1, v.ell, v.kmax, NS, B, Sw, lane, onsite, nullptr, v.eself);
                    if (lane == 0) sh_hh[warp] = hh;
                }
            }
            __syncthreads();
            // the candidates in order: CGS2 against this step's new vectors, breakdown, scale
            for (int s = 0; s < kWarpsPerAtom; ++s) {
                const int t = nb + s;                  // index of the new vector
                const bool mine = warp == s && m0 + s < sh_nueff && sh_ext && t < nu;
                if (mine) {
                    for (int pass = 0; pass < 2; ++pass) {
                        double c[kWarpsPerAtom - 1];
                        for (int q = 0; q < s; ++q) {
                            double part = 0.0;
                            for (int sl = 0; sl < NS; ++sl) {
                                const int p = sl * 32 + lane;
                                double2 w0, w1, v0, v1;
                                ld4(B + 4 * p, w0, w1);
                                ld4(SUb + (size_t)(nb + q) * vs + 4 * p, v0, v1);
                                part = fma4(v0, v1, w0, w1, part);
                            }
                            c[q] = warp_sum(part);
                        }
                        for (int sl = 0; sl < NS; ++sl) {
                            const int p = sl * 32 + lane;
                            double2 w0, w1, s0, s1;
                            ld4(B + 4 * p, w0, w1);
                            ld4(Sw + 4 * p, s0, s1);
                            for (int q = 0; q < s; ++q) {
                                double2 u0, u1, v0, v1;
                                ld4(Ub + (size_t)(nb + q) * vs + 4 * p, u0, u1);
                                ld4(SUb + (size_t)(nb + q) * vs + 4 * p, v0, v1);
                                w0.x = fma(-u0.x, c[q], w0.x); w0.y = fma(-u0.y, c[q], w0.y);
                                w1.x = fma(-u1.x, c[q], w1.x); w1.y = fma(-u1.y, c[q], w1.y);
                                s0.x = fma(-v0.x, c[q], s0.x); s0.y = fma(-v0.y, c[q], s0.y);
                                s1.x = fma(-v1.x, c[q], s1.x); s1.y = fma(-v1.y, c[q], s1.y);
                            }
                            st4(B + 4 * p, w0, w1);
                            st4(Sw + 4 * p, s0, s1);
                        }
                        __syncwarp();
                    }
                    double part = 0.0;
                    for (int sl = 0; sl < NS; ++sl) {
                        const int p = sl * 32 + lane;
                        double2 w0, w1, s0, s1;
                        ld4(B + 4 * p, w0, w1);
                        ld4(Sw + 4 * p, s0, s1);
                        part = fma4(w0, w1, s0, s1, part);
                    }
                    const double beta2 = warp_sum(part);
                    const double beta = sqrt(fmax(beta2, 0.0));
                    if (!(beta2 == beta2)) {
                        if (lane == 0) { flag(a.status, DEV_NONFINITE); sh_ext = 0; sh_nueff = t; }
                    } else if (beta2 < -(a.breakdown_tol * a.breakdown_tol) * sh_hh[warp]) {   // S not SPD
                        if (lane == 0) { flag(a.status, DEV_NOT_SPD); sh_ext = 0; sh_nueff = t; }
                    } else if (beta <= a.breakdown_tol * sqrt(sh_hh[warp])) {
                        if (lane == 0) { sh_ext = 0; sh_nueff = t; }
                    } else {
                        const double inv = 1.0 / beta;
                        for (int sl = 0; sl < NS; ++sl) {
                            const int p = sl * 32 + lane;
                            double2 w0, w1, s0, s1;
                            ld4(B + 4 * p, w0, w1);
                            ld4(Sw + 4 * p, s0, s1);
                            w0.x *= inv; w0.y *= inv; w1.x *= inv; w1.y *= inv;
                            s0.x *= inv; s0.y *= inv; s1.x *= inv; s1.y *= inv;
                            st4(Ub + (size_t)t * vs + 4 * p, w0, w1);
                            st4(SUb + (size_t)t * vs + 4 * p, s0, s1);
                        }
                        if (lane == 0) sh_nb = t + 1;
                    }
                }
                __syncthreads();
            }
            if (tid == 0 && sh_nb >= nu) sh_ext = 0;
            __syncthreads();
        }

        // ---------------------------------------------------------------- per-column outputs
        const int nu_eff = sh_nueff;
        if (tid < kWarpsPerAtom) {
            a.nu_eff[4 * J + tid] = nu_eff;
            if (nu_eff < nu) flag(a.status, DEV_BREAKDOWN);
        }
        if (a.UP) {   // pattern rows of U (the same basis for the 4 columns)
            const int alpha = warp;
            const int e0 = a.row_ptr[J], ne = a.row_ptr[J + 1] - e0;
            for (int q = lane; q < ne * 4; q += 32) {
                const int e = e0 + (q >> 2), r = q & 3;
                const int bb = bsearch_sorted(v.cl, n_at, a.col_idx[e]);
                const int p = v.pos_of[bb];
                double* out = a.UP + ((size_t)((e - a.up_block0) * 4 + alpha) * 4 + r) * nm;
                for (int k = 0; k < nu_eff; ++k) out[k] = Ub[4 * ((size_t)k * NP + p) + r];
            }
        }
        __syncthreads();
    }
}

size_t block_krylov_scratch_doubles(int nu_max, int na_max) {
    return (size_t)(2 * nu_max + kWarpsPerAtom) * na_max * 4;
}

int block_krylov_blocks_per_sm(int na_max, int deg_max) {
    const size_t smem = krylov_smem_bytes(na_max, deg_max);
    smem_at_least(k_block_krylov, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_block_krylov, kThreads, smem);
    return nb;
}

void block_krylov_columns(const KrylovArgs& a, int grid, cudaStream_t st) {
    const size_t smem = krylov_smem_bytes(a.na_max, a.deg_max);
    smem_at_least(k_block_krylov, smem);
    k_block_krylov<<<grid, kThreads, smem, st>>>(a);
}

}  // namespace elses
