// Exact gradient of the grand potential through the truncated Krylov build: dOmega/dH and
// dOmega/dS on the BSR pattern, for the columns of a batch of atoms.
//
// Omega = sum_j Omega_j at fixed mu, Omega_j = sum_k d_k c_k w(e_k) with w the grand-potential
// weight of the Fermi-Dirac occupation (w' = 2 f). The density-matrix adjoint
// (dOmega/dH = rho, dOmega/dS = -rhoE) is its gradient only when the Krylov space spans the
// cluster; at a truncated nu the space K_nu(H_C, e_j) moves with H. Per column, with U the
// S-orthonormal basis, H' = U^T H U, S' = U^T S U = I, a = U^T e_j, b = U^T S e_j
// (= sqrt(S_jj) e_1) and Omega_j = b^T w(H') a:
//
//  1. Rayleigh-Ritz at a fixed basis. With H' = Q diag(e) Q^T (Q: the eigenvectors V of the
//     projected problem), c = Q^T a, d = Q^T b:
//       Hh   = dOmega/dH' = Q (Gamma o sym(d c^T)) Q^T, Gamma the divided differences of w
//              (Daleckii-Krein; Gamma_kk = w'(e_k) = 2 f(e_k)),
//       abar = dOmega/da = Q (w o d),  bbar = dOmega/db = Q (w o c),
//       Sh   = dOmega/dS' = -H' Hh - (a abar^T + b bbar^T) / 2 (Omega is unchanged by a change
//              of basis U -> U M, which fixes dOmega/dS' once the others are known),
//     so that, at a fixed U, dOmega/dH = U Hh U^T, dOmega/dS = U Sh U^T + e_j (U bbar)^T (b is
//     read from row j of S U) and
//       G_U = dOmega/dU = 2 HU Hh + 2 SU Sh + e_j abar^T + S e_j bbar^T  (U^T G_U = 0).
//  2. The space moves with H only. Reverse mode of the Gram-Schmidt recursion
//     h_n = H u_n, a_n = U_n^T S h_n, w_n = h_n - U_n a_n, beta_n = |w_n|_S, u_{n+1} = w_n / beta_n
//     seeded with Ubar = G_U, for n = nu - 1 .. 1:
//       bb = -(ubar_{n+1} . u_{n+1}) / beta_n,   wbar = ubar_{n+1} / beta_n + bb S u_{n+1},
//       abar_n = -U_n^T wbar,   hbar_n = wbar + S U_n abar_n,
//       Ubar_{1..n} += -wbar a_n^T + (S h_n) abar_n^T   with S h_n = SU_{n+1} [a_n; beta_n],
//       dOmega/dH += hbar_n u_n^T,   ubar_n += H hbar_n.
//     Its S terms, the scale of the start u_1 = e_j / sqrt(S_jj) among them, add up to zero:
//     S only changes the basis inside the space, and U^T G_U = 0. (They are left out rather
//     than summed: with a nearly exhausted space the 1 / beta factors would amplify their
//     rounding.)
//  So dOmega/dH = Y_H U^T and dOmega/dS = Y_S U^T with n_c x nu factors
//       Y_H = U Hh + [hbar_1 .. hbar_{nu-1}, 0],
//       Y_S = U Sh + e_j bbar^T,
//  sampled on the blocks of the cluster (the 4 columns of the atom summed) and added atomically
//  into per-entry accumulators. Each contribution is taken exactly (to 2^-80) into a 128-bit
//  fixed-point integer and added as two 64-bit words with the carry: integer addition is
//  associative, so the sums, and the gradient and forces after them, are the same bit for bit
//  whatever the order in which the CTAs arrive. One pass at the end converts them to FP64.
//
// The bases come from the energy pass when it kept them (the Krylov kernel's store form),
// otherwise the forward recursion is recomputed here by the Krylov kernel's own code
// (column_forward with kAdj: it also keeps HU and the Gram-Schmidt coefficients); V, e, c, d
// come from the columns already computed for the same positions. One CTA of 4 warps per atom; the lanes own cluster
// rows as in the Krylov kernel; the bases and factors live in per-warp global scratch.
#include "krylov.cuh"

namespace elses {

namespace {

// (w(x) - w(y)) / (x - y), and w'(x) = 2 f(x) at x = y. For |x - y| <= kT the difference is
// taken in the exact form w(x) - w(y) = -2 kT log1p(f(y) expm1(-(x - y)/kT)), which does not
// cancel.
__device__ __forceinline__ double omega_divdiff(double x, double y, double wx, double wy, double fy,
                                                double kT) {
    if (x == y) return 2.0 * fy;
    const double dx = (x - y) / kT;
    if (fabs(dx) > 1.0) return (wx - wy) / (x - y);
    return -2.0 * kT * log1p(fy * expm1(-dx)) / (x - y);
}

// ---- exact fixed-point accumulation: value * 2^80 as a 128-bit two's complement integer
constexpr int kFixFrac = 80;                 // fractional bits (resolution 8e-25)

// The 128-bit integer of v * 2^80, truncated toward zero below 2^-80. |v| < 2^46 (far above any
// gradient entry); a larger or non-finite v sets DEV_NONFINITE and adds nothing.
__device__ __forceinline__ bool to_fixed(double v, unsigned long long& lo, unsigned long long& hi) {
    const long long bits = __double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    lo = hi = 0ull;
    if (ex == 0) return true;                                        // zero or subnormal
    const int shift = ex - 1075 + kFixFrac;                          // v = mant * 2^(ex - 1075)
    if (ex == 0x7ff || shift > 127 - 53 - 1) return false;
    unsigned __int128 m = (unsigned long long)(bits & ((1ll << 52) - 1)) | (1ull << 52);
    if (shift >= 0) m <<= shift;
    else m = shift <= -64 ? (unsigned __int128)0 : (m >> -shift);
    if (bits < 0) m = (unsigned __int128)0 - m;
    lo = (unsigned long long)m;
    hi = (unsigned long long)(m >> 64);
    return true;
}

// p[0] (low word) and p[1] (high word) += (lo, hi): the low words add modulo 2^64 and the carry
// out of each addition goes to the high word, so the pair ends as the exact 128-bit sum.
__device__ __forceinline__ void fixed_add(unsigned long long* p, double v, int* status) {
    unsigned long long lo, hi;
    if (!to_fixed(v, lo, hi)) {
        flag(status, DEV_NONFINITE);
        return;
    }
    if (lo) {
        const unsigned long long old = atomicAdd(p, lo);
        hi += (old + lo < old) ? 1ull : 0ull;
    }
    if (hi) atomicAdd(p + 1, hi);
}

__global__ void k_fixed_to_double(const unsigned long long* __restrict__ acc, size_t n, double s_scale,
                                  double* __restrict__ gH, double* __restrict__ gS) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 2 * n; q += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long lo = acc[2 * q], hi = acc[2 * q + 1];
        const bool neg = (long long)hi < 0;
        unsigned __int128 m = ((unsigned __int128)hi << 64) | lo;
        if (neg) m = (unsigned __int128)0 - m;
        const double d = __ull2double_rn((unsigned long long)(m >> 64)) * 18446744073709551616.0 +
                         __ull2double_rn((unsigned long long)m);
        const double v = ldexp(neg ? -d : d, -kFixFrac);
        if (q < n) gH[q] = v;
        else gS[q - n] = s_scale * v;
    }
}

// packed upper storage of H' (element (i, k), i <= k, at i + k (k + 1) / 2)
__device__ __forceinline__ double packed_at(const double* P, int i, int k) {
    return i <= k ? P[i + k * (k + 1) / 2] : P[k + i * (i + 1) / 2];
}

struct WarpScratch {
    double *U, *SU, *HU, *Ub, *YH, *YS, *T;        // vectors: nm x (NA x 4) each, T: NA x 4
    double *hess, *X, *Tm, *Hh, *Sg, *Sy;           // nm x nm each
    double *om, *abar, *bbar;                      // nm each
};

__device__ __forceinline__ WarpScratch warp_scratch(double* base, int nm, int NA) {
    WarpScratch w;
    const size_t vsz = (size_t)nm * NA * 4, mm = (size_t)nm * nm;
    w.U = base;
    w.SU = w.U + vsz;
    w.HU = w.SU + vsz;
    w.Ub = w.HU + vsz;
    w.YH = w.Ub + vsz;
    w.YS = w.YH + vsz;
    w.T = w.YS + vsz;
    w.hess = w.T + (size_t)NA * 4;
    w.X = w.hess + mm;
    w.Tm = w.X + mm;
    w.Hh = w.Tm + mm;
    w.Sg = w.Hh + mm;
    w.Sy = w.Sg + mm;
    w.om = w.Sy + mm;
    w.abar = w.om + nm;
    w.bbar = w.abar + nm;
    return w;
}

// Step 1 for one column (lanes over entries of the small matrices): Hh, abar, bbar, Sh (into
// Sy) and the form of Sh that G_U takes (Sg: row 1 += sqrt(S_jj) bbar^T / 2, the S e_j bbar^T
// term with S e_j = sqrt(S_jj) SU_1).
__device__ __forceinline__ void rayleigh_ritz_gradient(const AdjointArgs& g, const double* Vc, const double* ec,
                                                       const double* cc, const double* dc, const double* Hpc,
                                                       const WarpScratch& w, int nv, int nm, size_t vs, int jp,
                                                       double sq, int lane) {
    const double mu = g.mu_dev ? *g.mu_dev : g.mu;
    for (int k = lane; k < nv; k += 32) w.om[k] = omega_w(ec[k], mu, g.kT);
    __syncwarp();
    for (int q = lane; q < nv * nv; q += 32) {
        const int k = q / nv, l = q % nv;
        const double G = omega_divdiff(ec[k], ec[l], w.om[k], w.om[l], fermi((ec[l] - mu) / g.kT), g.kT);
        w.X[k * nm + l] = G * 0.5 * (dc[k] * cc[l] + cc[k] * dc[l]);
    }
    __syncwarp();
    for (int q = lane; q < nv * nv; q += 32) {       // Tm = X V^T
        const int k = q / nv, n = q % nv;
        double s = 0.0;
        for (int l = 0; l < nv; ++l) s = fma(w.X[k * nm + l], Vc[n * nm + l], s);
        w.Tm[k * nm + n] = s;
    }
    __syncwarp();
    for (int q = lane; q < nv * nv; q += 32) {       // Hh = V Tm
        const int n = q / nv, m = q % nv;
        double s = 0.0;
        for (int k = 0; k < nv; ++k) s = fma(Vc[n * nm + k], w.Tm[k * nm + m], s);
        w.Hh[n * nm + m] = s;
    }
    for (int n = lane; n < nv; n += 32) {            // abar = V (w o d), bbar = V (w o c)
        double s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < nv; ++k) {
            const double t = Vc[n * nm + k] * w.om[k];
            s1 = fma(t, dc[k], s1);
            s2 = fma(t, cc[k], s2);
        }
        w.abar[n] = s1;
        w.bbar[n] = s2;
    }
    __syncwarp();
    for (int q = lane; q < nv * nv; q += 32) {       // Sh = -H' Hh - (a abar^T + b bbar^T) / 2
        const int k = q / nv, n = q % nv;
        double s = 0.0;
        for (int m = 0; m < nv; ++m) s = fma(packed_at(Hpc, k, m), w.Hh[m * nm + n], s);
        const double ak = w.U[(size_t)k * vs + jp], bk = w.SU[(size_t)k * vs + jp];
        const double sh = -s - 0.5 * (ak * w.abar[n] + bk * w.bbar[n]);
        w.Sg[k * nm + n] = sh + (k == 0 ? 0.5 * sq * w.bbar[n] : 0.0);
        w.Sy[k * nm + n] = sh;
    }
    __syncwarp();
}

// out[n] = sum_k X[k] C1[k][n] (+ Y[k] C2[k][n]) on the lane's rows of slot position p, four n at
// a time; `fin` finishes and stores each output vector.
template <bool kTwo, typename Fin>
__device__ __forceinline__ void combine(const double* X, const double* C1, const double* Y, const double* C2,
                                        int nv, int nm, size_t vs, int p, Fin fin) {
    for (int n0 = 0; n0 < nv; n0 += 4) {
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0;
        for (int k = 0; k < nv; ++k) {
            double2 x0, x1, y0, y1;
            ld4(X + (size_t)k * vs + 4 * p, x0, x1);
            if constexpr (kTwo) ld4(Y + (size_t)k * vs + 4 * p, y0, y1);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (n0 + i < nv) {
                    const double c1 = C1[k * nm + n0 + i];
                    acc[i][0] = fma(x0.x, c1, acc[i][0]);
                    acc[i][1] = fma(x0.y, c1, acc[i][1]);
                    acc[i][2] = fma(x1.x, c1, acc[i][2]);
                    acc[i][3] = fma(x1.y, c1, acc[i][3]);
                    if constexpr (kTwo) {
                        const double c2 = C2[k * nm + n0 + i];
                        acc[i][0] = fma(y0.x, c2, acc[i][0]);
                        acc[i][1] = fma(y0.y, c2, acc[i][1]);
                        acc[i][2] = fma(y1.x, c2, acc[i][2]);
                        acc[i][3] = fma(y1.y, c2, acc[i][3]);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (n0 + i < nv) fin(n0 + i, acc[i]);
    }
}

// Step 2: the reverse Gram-Schmidt sweep (lanes over rows; A, B: the warp's shared vectors,
// hb: its coefficient buffer). Leaves hbar_n in YH[n] (n <= nv - 2) and the final Ubar.
__device__ __forceinline__ void reverse_sweep(const KrylovArgs& a, const ClusterView& v, const WarpScratch& w,
                                              double* A, double* B, double* hb, int nv, int nm, size_t vs,
                                              int lane) {
    const int NS = v.NS;
    const bool onsite = a.onsite_diag != 0;
    for (int m = nv - 2; m >= 0; --m) {
        const double* am = w.hess + (size_t)m * nm;        // a_m[k], k <= m; beta_m at m + 1
        const double beta = am[m + 1];
        const double* Um1 = w.U + (size_t)(m + 1) * vs;
        const double* SUm1 = w.SU + (size_t)(m + 1) * vs;
        const double* ubm1 = w.Ub + (size_t)(m + 1) * vs;
        double part = 0.0;
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * 32 + lane;
            double2 x0, x1, u0, u1;
            ld4(ubm1 + 4 * p, x0, x1);
            ld4(Um1 + 4 * p, u0, u1);
            part = fma4(x0, x1, u0, u1, part);
        }
        const double ib = 1.0 / beta;
        const double bb = -warp_sum(part) * ib;
        // wbar (into A) and abar_m = -U_{0..m}^T wbar, sixteen k at a time
        for (int k0 = 0; k0 <= m; k0 += 16) {
            double acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.0;
            for (int sl = 0; sl < NS; ++sl) {
                const int p = sl * 32 + lane;
                double2 w0, w1;
                if (k0 == 0) {
                    double2 x0, x1, s0, s1;
                    ld4(ubm1 + 4 * p, x0, x1);
                    ld4(SUm1 + 4 * p, s0, s1);
                    w0 = make_double2(fma(bb, s0.x, x0.x * ib), fma(bb, s0.y, x0.y * ib));
                    w1 = make_double2(fma(bb, s1.x, x1.x * ib), fma(bb, s1.y, x1.y * ib));
                    st4(A + 4 * p, w0, w1);
                } else {
                    ld4(A + 4 * p, w0, w1);
                }
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    if (k0 + kk <= m) {
                        double2 u0, u1;
                        ld4(w.U + (size_t)(k0 + kk) * vs + 4 * p, u0, u1);
                        acc[kk] = fma4(u0, u1, w0, w1, acc[kk]);
                    }
                }
            }
            const double r = warp_sum16(acc);
            __syncwarp();
            if (lane < 16 && k0 + lane <= m) hb[k0 + lane] = -r;
            __syncwarp();
        }
        // hbar = wbar + SU_{0..m} abar (into B and YH[m]); S h_m; Ubar_{0..m} update
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * 32 + lane;
            double2 w0, w1;
            ld4(A + 4 * p, w0, w1);
            double2 h0 = w0, h1 = w1, s0 = make_double2(0.0, 0.0), s1 = s0;
            for (int k = 0; k <= m + 1; ++k) {
                double2 x0, x1;
                ld4(w.SU + (size_t)k * vs + 4 * p, x0, x1);
                const double ck = am[k];
                s0.x = fma(x0.x, ck, s0.x); s0.y = fma(x0.y, ck, s0.y);
                s1.x = fma(x1.x, ck, s1.x); s1.y = fma(x1.y, ck, s1.y);
                if (k <= m) {
                    const double ak = hb[k];
                    h0.x = fma(x0.x, ak, h0.x); h0.y = fma(x0.y, ak, h0.y);
                    h1.x = fma(x1.x, ak, h1.x); h1.y = fma(x1.y, ak, h1.y);
                }
            }
            st4(B + 4 * p, h0, h1);
            st4(w.YH + (size_t)m * vs + 4 * p, h0, h1);
            for (int k = 0; k <= m; ++k) {
                double2 x0, x1;
                double* ub = w.Ub + (size_t)k * vs + 4 * p;
                ld4(ub, x0, x1);
                const double ck = -am[k], ak = hb[k];
                x0.x = fma(w0.x, ck, fma(s0.x, ak, x0.x)); x0.y = fma(w0.y, ck, fma(s0.y, ak, x0.y));
                x1.x = fma(w1.x, ck, fma(s1.x, ak, x1.x)); x1.y = fma(w1.y, ck, fma(s1.y, ak, x1.y));
                st4(ub, x0, x1);
            }
        }
        __syncwarp();
        // ubar_m += H hbar_m
        spmv(a.H, a.skr, 0, v.ell, v.kmax, NS, B, w.T, lane, onsite, a.H, v.eself);
        for (int sl = 0; sl < NS; ++sl) {
            const int p = sl * 32 + lane;
            double2 x0, x1, t0, t1;
            double* ub = w.Ub + (size_t)m * vs + 4 * p;
            ld4(ub, x0, x1);
            ld4(w.T + 4 * p, t0, t1);
            x0.x += t0.x; x0.y += t0.y; x1.x += t1.x; x1.y += t1.y;
            st4(ub, x0, x1);
        }
        __syncwarp();
    }
}

// dOmega/dH and dOmega/dS of block blk between cluster rows at rp4 = 4 p and columns at
// cp4 = 4 p': sum over the atom's columns and n of Y[p][a][n] U[p'][b][n] (Uw, YHw, YSw: the
// warps' bases and factors).
__device__ __forceinline__ void sampled_block(const AdjointArgs& g, const int* nvw, const double* const* Uw,
                                              const double* const* YHw, const double* const* YSw, size_t vs,
                                              int rp4, int cp4, int blk) {
    double aH[16], aS[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) { aH[q] = 0.0; aS[q] = 0.0; }
    for (int wi = 0; wi < kWarpsPerAtom; ++wi) {
        const double* U = Uw[wi];
        const double* YH = YHw[wi];
        const double* YS = YSw[wi];
        for (int n = 0; n < nvw[wi]; ++n) {
            double2 x0, x1, y0, y1, z0, z1;
            ld4(U + (size_t)n * vs + cp4, x0, x1);
            ld4(YH + (size_t)n * vs + rp4, y0, y1);
            ld4(YS + (size_t)n * vs + rp4, z0, z1);
            const double xs[4] = {x0.x, x0.y, x1.x, x1.y};
            const double ys[4] = {y0.x, y0.y, y1.x, y1.y};
            const double zs[4] = {z0.x, z0.y, z1.x, z1.y};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    aH[4 * r + c] = fma(ys[r], xs[c], aH[4 * r + c]);
                    aS[4 * r + c] = fma(zs[r], xs[c], aS[4 * r + c]);
                }
        }
    }
    unsigned long long* oH = g.acc + 2 * 16 * (size_t)blk;
    unsigned long long* oS = oH + 2 * 16 * (size_t)g.nnzb;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        fixed_add(oH + 2 * q, aH[q], g.status);
        fixed_add(oS + 2 * q, aS[q], g.status);
    }
}

}  // namespace

__host__ __device__ size_t adjoint_warp_doubles(int nm, int na_max) {
    const size_t d = 6 * (size_t)nm * na_max * 4 + (size_t)na_max * 4 + 6 * (size_t)nm * nm + 3 * (size_t)nm;
    return (d + 3) & ~(size_t)3;   // keeps every warp's area 32-byte aligned
}

// Register cap for 3 CTAs per SM (168 registers, a few hundred bytes of spills to L1-cached local
// memory): 12 warps per SM hide the basis reads better than 8 at 254 registers. Measured on the
// 4096-atom exact-force step: 201.7 -> 186.9 ms.
__global__ void __launch_bounds__(kThreads, 3) k_adjoint(const KrylovArgs a, const AdjointArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NA = a.na_max, nm = a.nu_max;
    double* vec = reinterpret_cast<double*>(smem_raw);
    double* hbuf = vec + (size_t)kWarpsPerAtom * 2 * NA * 4;
    ClusterView v;
    carve_view(reinterpret_cast<unsigned char*>(hbuf + kWarpsPerAtom * kMaxNu), NA, a.deg_max, v);
    __shared__ int sh_atom, sh_nv[kWarpsPerAtom];
    __shared__ const double* sh_U[kWarpsPerAtom];
    __shared__ const double* sh_YH[kWarpsPerAtom];
    __shared__ const double* sh_YS[kWarpsPerAtom];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const WarpScratch ws =
        warp_scratch(g.scratch + ((size_t)blockIdx.x * kWarpsPerAtom + warp) * adjoint_warp_doubles(nm, NA), nm, NA);

    for (int iter = 0;; ++iter) {
        if (tid == 0) {
            const int idx = a.queue ? atomicAdd(a.queue, 1) : blockIdx.x + iter * gridDim.x;
            int atom = -1;
            if (idx < a.n_items) {
                atom = a.order[idx];
                if (atom < g.atom_lo || atom >= g.atom_hi) atom = -2;   // outside the requested atoms
            }
            sh_atom = atom;
        }
        __syncthreads();
        const int J = sh_atom;
        if (J == -1) break;
        if (J < 0) {
            __syncthreads();
            continue;
        }
        if (!cluster_view(a, J, NA, v)) {
            if (tid == 0) flag(a.status, DEV_CAPACITY);
            __syncthreads();
            continue;
        }
        const size_t vs = (size_t)v.NS * 32 * 4;
        int nv = 0;
        WarpScratch w = ws;
        do {
            const int alpha = warp, j = 4 * J + alpha;
            double* A = vec + (size_t)(warp * 2) * NA * 4;
            double* B = A + (size_t)NA * 4;
            double* hb = hbuf + warp * kMaxNu;
            int jp = 0;
            const double* Hpc;
            if (g.bstore) {   // the bases the energy pass kept
                const int aJ = bsearch_sorted(v.cl, v.n_at, J);
                nv = aJ >= 0 ? a.nu_eff[j] : 0;
                if (nv <= 0) {
                    nv = 0;
                    break;
                }
                jp = 4 * v.pos_of[aJ] + alpha;
                double* col = const_cast<double*>(g.bstore) + (size_t)j * g.bstride;
                w.U = col;
                w.SU = col + g.bvec;
                w.HU = col + 2 * g.bvec;
                w.hess = col + 3 * g.bvec;
                Hpc = w.hess + (size_t)nm * nm;
            } else {
                int nu = 0;
                nv = column_forward<true>(a, v, J, alpha, A, B, hb, w.U, w.SU, w.HU, w.hess, nu, jp);
                if (nv <= 0) {
                    nv = 0;
                    break;
                }
                Hpc = a.Hp + (size_t)(j - 4 * a.atom_begin) * (nm * (nm + 1) / 2);
            }
            __syncwarp();
            const double sq = 1.0 / w.U[jp];                   // sqrt(S_jj): u_1 = e_j / sqrt(S_jj)
            rayleigh_ritz_gradient(g, g.V + (size_t)(j - g.v_col0) * nm * nm, g.eps + (size_t)j * nm,
                                   g.c + (size_t)j * nm, g.d + (size_t)j * nm, Hpc, w, nv, nm, vs, jp, sq, lane);
            // G_U = 2 (HU Hh + SU Sg) + e_j abar^T into Ubar
            for (int sl = 0; sl < v.NS; ++sl) {
                const int p = sl * 32 + lane;
                combine<true>(w.HU, w.Hh, w.SU, w.Sg, nv, nm, vs, p, [&](int n, const double* s) {
                    double o[4] = {2.0 * s[0], 2.0 * s[1], 2.0 * s[2], 2.0 * s[3]};
                    const int r = jp - 4 * p;
                    if (r >= 0 && r < 4) o[r] += w.abar[n];
                    st4(w.Ub + (size_t)n * vs + 4 * p, make_double2(o[0], o[1]), make_double2(o[2], o[3]));
                });
            }
            __syncwarp();
            reverse_sweep(a, v, w, A, B, hb, nv, nm, vs, lane);
            // Y_H = U Hh + [hbar ..., 0];  Y_S = U Sh + e_j bbar^T
            for (int sl = 0; sl < v.NS; ++sl) {
                const int p = sl * 32 + lane;
                combine<false>(w.U, w.Hh, nullptr, nullptr, nv, nm, vs, p, [&](int n, const double* s) {
                    double2 h0 = make_double2(0.0, 0.0), h1 = h0;
                    if (n < nv - 1) ld4(w.YH + (size_t)n * vs + 4 * p, h0, h1);
                    st4(w.YH + (size_t)n * vs + 4 * p, make_double2(h0.x + s[0], h0.y + s[1]),
                        make_double2(h1.x + s[2], h1.y + s[3]));
                });
                combine<false>(w.U, w.Sy, nullptr, nullptr, nv, nm, vs, p, [&](int n, const double* s) {
                    double o[4] = {s[0], s[1], s[2], s[3]};
                    const int r = jp - 4 * p;
                    if (r >= 0 && r < 4) o[r] += w.bbar[n];
                    st4(w.YS + (size_t)n * vs + 4 * p, make_double2(o[0], o[1]), make_double2(o[2], o[3]));
                });
            }
        } while (0);
        if (lane == 0 && g.flops && nv > 0) {
            // algorithmic flops of this column (formula in include/elses.h, elses_stats)
            const unsigned long long vv = nv, nc = 4ull * v.n_at, nent = v.nent, nat = v.n_at;
            const bool onsite = a.onsite_diag != 0;
            const unsigned long long per = a.skr ? 24ull : 32ull;
            const unsigned long long blocks = nent + (onsite ? nat : 0ull);
            unsigned long long f = 8ull * vv * vv * nc + 6ull * vv * vv * vv + 64ull * vv * blocks;
            f += (vv - 1) * (8ull * nc + per * nent + (onsite ? 4ull * nat : 0ull)) + 5ull * nc * vv * (vv - 1);
            if (!g.bstore)   // the forward recursion recomputed: the Krylov kernel's count
                f += column_flops(a, v.n_at, v.nent, nv, a.reorth != 0);
            atomicAdd(g.flops, f);
        }
        if (lane == 0) {
            sh_nv[warp] = nv;
            sh_U[warp] = w.U;
            sh_YH[warp] = w.YH;
            sh_YS[warp] = w.YS;
        }
        __syncthreads();
        // sampled products over the cluster's blocks: lane l's list entries, every 4th from `warp`
        for (int k = warp; k < v.kmax; k += kWarpsPerAtom) {
            const Ent en = v.ell[32 * k + lane];
            if (en.blk < 0) continue;
            const int p = (en.p4 >> 16) * 32 + lane;
            sampled_block(g, sh_nv, sh_U, sh_YH, sh_YS, vs, 4 * p, en.p4 & 0xffff, en.blk);
        }
        if (a.onsite_diag) {   // on-site blocks are not list entries then
            for (int sl = warp; sl < v.NS; sl += kWarpsPerAtom) {
                const int p = sl * 32 + lane;
                const int es = v.eself[p];
                if (es >= 0) sampled_block(g, sh_nv, sh_U, sh_YH, sh_YS, vs, 4 * p, 4 * p, es);
            }
        }
        __syncthreads();
    }
}

int adjoint_blocks_per_sm(int na_max, int deg_max) {
    const size_t smem = krylov_smem_bytes(na_max, deg_max);
    smem_at_least(k_adjoint, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint, kThreads, smem);
    return nb;
}

void adjoint_finish(const unsigned long long* acc, size_t n, double s_scale, double* gH, double* gS,
                    cudaStream_t st) {
    const int threads = 256;
    const int grid = (int)std::min<size_t>((2 * n + threads - 1) / threads, 152 * 16);
    k_fixed_to_double<<<std::max(grid, 1), threads, 0, st>>>(acc, n, s_scale, gH, gS);
}

void adjoint_columns(const KrylovArgs& a, const AdjointArgs& g, int grid, cudaStream_t st) {
    const size_t smem = krylov_smem_bytes(a.na_max, a.deg_max);
    smem_at_least(k_adjoint, smem);
    k_adjoint<<<grid, kThreads, smem, st>>>(a, g);
}

}  // namespace elses
