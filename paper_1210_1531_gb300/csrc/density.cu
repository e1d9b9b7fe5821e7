// a8: density-matrix columns on the pattern; G_ij(z) on the pattern for given z.
//
// Eq. 2: rho_ij = -(1/pi) Int f(e - mu) Im G_ij(e + i0) de. With G_ij(z) = sum_k Z_ik c_k /
// (z - e_k) the integral is taken by residues (Im 1/(e + i0 - e_k) = -pi delta(e - e_k)):
//     rho_ij  = 2 sum_k f(e_k - mu) Z_ik c_k          (2: spin)
//     rhoE_ij = 2 sum_k f(e_k - mu) e_k Z_ik c_k
// for the pattern rows i of column j (atoms within r_cut of J), with Z = U V. Computed as
// t = V (2 f c) (nu x nu) followed by rho_P = U_P t, which needs no Z. Where V is not formed, t
// comes from the eigen-factors: V w = L^-T Q_H (R_1^T .. R_n^T w), the rotations applied by
// k_eig_weights, the reflectors and L^-T here.
//
// One CTA per atom J, one warp per column; column j = 4J + b writes rho[(I, J)][a][b] through
// the transpose map of the pattern (each element is written exactly once).
#include "internal.h"

namespace elses {

// Two warp-wide sums at once (recursive halving, then a butterfly within each half): 5 additions
// instead of 10. Both sums are returned in every lane.
__device__ __forceinline__ void warp_sum_pair(double& x, double& y) {
    const int lane = threadIdx.x & 31;
    const bool upper = lane & 16;
    double v = (upper ? y : x) + __shfl_xor_sync(0xffffffffu, upper ? x : y, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    x = __shfl_sync(0xffffffffu, v, 0);
    y = __shfl_sync(0xffffffffu, v, 16);
}

// t = L^-T Q_H u for the pair (u, u_E) of column j from the kept eigen-factors: the reflectors
// H_{nu-3} .. H_0 (H_k x = x - tau_k v_k v_k^T x, v_k in row k of the first factor matrix), then
// the back substitution with L^T. Lanes over rows (row lane, and lane + 32 when nu > 32).
template <bool kTwo>
__device__ __forceinline__ void apply_factors(const DensityArgs& a, int j, int nu, double* t, double* tE) {
    const int lane = threadIdx.x & 31, nm = a.nu_max;
    const double* F = a.fac + (size_t)(j - a.v_col0) * 2 * nm * nm;
    const double* Lf = F + (size_t)nm * nm;
    const double* u = a.T + (size_t)(j - a.v_col0) * 2 * nm;
    const int r1 = lane + 32;
    double x0 = 0.0, e0 = 0.0, x1 = 0.0, e1 = 0.0;   // zero past nu
    if (lane < nm) { x0 = u[lane]; e0 = u[nm + lane]; }
    if (kTwo && r1 < nm) { x1 = u[r1]; e1 = u[nm + r1]; }
    for (int k = nu - 3; k >= 0; --k) {
        const double* v = F + (size_t)k * nm;
        const double tau = v[k];
        if (tau == 0.0) continue;
        const double v0 = (lane > k && lane < nu) ? v[lane] : 0.0;
        const double v1 = (kTwo && r1 > k && r1 < nu) ? v[r1] : 0.0;
        double s = v0 * x0, sE = v0 * e0;
        if (kTwo) { s = fma(v1, x1, s); sE = fma(v1, e1, sE); }
        warp_sum_pair(s, sE);
        s *= tau;
        sE *= tau;
        x0 = fma(-s, v0, x0);
        e0 = fma(-sE, v0, e0);
        if (kTwo) { x1 = fma(-s, v1, x1); e1 = fma(-sE, v1, e1); }
    }
    // L^T t = x, bottom-up: t_i = x_i / L_ii, then x_l -= L_il t_i for l < i
    const double i0 = lane < nu ? 1.0 / Lf[(size_t)lane * nm + lane] : 0.0;
    const double i1 = (kTwo && r1 < nu) ? 1.0 / Lf[(size_t)r1 * nm + r1] : 0.0;
    for (int i = nu - 1; i >= 0; --i) {
        const bool hi = kTwo && i >= 32;
        const int owner = i & 31;
        const double ti = __shfl_sync(0xffffffffu, hi ? x1 * i1 : x0 * i0, owner);
        const double tEi = __shfl_sync(0xffffffffu, hi ? e1 * i1 : e0 * i0, owner);
        const double* row = Lf + (size_t)i * nm;
        const double l0 = lane < i ? row[lane] : 0.0;
        x0 = lane == i ? ti : fma(-l0, ti, x0);
        e0 = lane == i ? tEi : fma(-l0, tEi, e0);
        if (kTwo) {
            const double l1 = r1 < i ? row[r1] : 0.0;
            x1 = r1 == i ? ti : fma(-l1, ti, x1);
            e1 = r1 == i ? tEi : fma(-l1, tEi, e1);
        }
    }
    if (lane < nu) { t[lane] = x0; tE[lane] = e0; }
    if (kTwo && r1 < nu) { t[r1] = x1; tE[r1] = e1; }
}

__global__ void __launch_bounds__(128) k_density(const DensityArgs a) {
    __shared__ double wc[4][kMaxNu], wec[4][kMaxNu], t[4][kMaxNu], tE[4][kMaxNu];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int J = a.atom_begin + blockIdx.x;
    if (J >= a.atom_end) return;
    const int j = 4 * J + warp;
    const int nm = a.nu_max;
    const int nu = a.nu_eff[j];
    if (a.T) {
        if (nu > 32) apply_factors<true>(a, j, nu, t[warp], tE[warp]);
        else apply_factors<false>(a, j, nu, t[warp], tE[warp]);
    } else {
        for (int k = lane; k < nu; k += 32) {
            const double e = a.eps[(size_t)j * nm + k];
            const double f2 = 2.0 * fermi((e - a.mu) / a.kT) * a.c[(size_t)j * nm + k];
            wc[warp][k] = f2;
            wec[warp][k] = f2 * e;
        }
        __syncwarp();
        const double* V = a.V + (size_t)(j - a.v_col0) * nm * nm;
        for (int n = lane; n < nu; n += 32) {
            double s = 0.0, sE = 0.0;
            for (int k = 0; k < nu; ++k) {
                const double v = V[(size_t)n * nm + k];
                s += v * wc[warp][k];
                sE += v * wec[warp][k];
            }
            t[warp][n] = s;
            tE[warp][n] = sE;
        }
    }
    __syncwarp();
    const int e0 = a.row_ptr[J], ne = a.row_ptr[J + 1] - e0;
    for (int q = lane; q < ne * 4; q += 32) {
        const int e = e0 + (q >> 2), r = q & 3;
        const double* up = a.UP + ((size_t)((e - a.up_block0) * 4 + warp) * 4 + r) * nm;
        double s = 0.0, sE = 0.0;
        for (int k = 0; k < nu; ++k) {
            s += up[k] * t[warp][k];
            sE += up[k] * tE[warp][k];
        }
        const int et = a.tmap[e];
        if (et < 0) continue;   // the pattern is symmetric by construction; never taken
        const size_t o = 16 * (size_t)et + 4 * r + warp;
        a.rho[o] = s;
        if (a.rhoE) a.rhoE[o] = sE;
    }
}

void density_columns(const DensityArgs& a, cudaStream_t st) {
    const int n = a.atom_end - a.atom_begin;
    if (n > 0) k_density<<<n, 128, 0, st>>>(a);
}

// G_ij(z) = sum_k Z_ik c_k / (z - e_k) on the pattern rows, for each z of the list.
__global__ void __launch_bounds__(128) k_green(const DensityArgs a) {
    __shared__ double tr[4][kMaxNu], ti[4][kMaxNu];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int J = a.atom_begin + blockIdx.x;
    if (J >= a.atom_end) return;
    const int j = 4 * J + warp;
    const int nm = a.nu_max;
    const int nu = a.nu_eff[j];
    const double* V = a.V + (size_t)(j - a.v_col0) * nm * nm;
    const int e0 = a.row_ptr[J], ne = a.row_ptr[J + 1] - e0;
    for (int iz = 0; iz < a.n_z; ++iz) {
        const double zr = a.z[2 * iz], zi = a.z[2 * iz + 1];
        for (int n = lane; n < nu; n += 32) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < nu; ++k) {
                const double ck = a.c[(size_t)j * nm + k];
                const double dr = zr - a.eps[(size_t)j * nm + k], di = zi;
                const double inv = 1.0 / (dr * dr + di * di);
                const double v = V[(size_t)n * nm + k] * ck;
                sr += v * dr * inv;
                si -= v * di * inv;
            }
            tr[warp][n] = sr;
            ti[warp][n] = si;
        }
        __syncwarp();
        for (int q = lane; q < ne * 4; q += 32) {
            const int e = e0 + (q >> 2), r = q & 3;
            const double* up = a.UP + ((size_t)((e - a.up_block0) * 4 + warp) * 4 + r) * nm;
            double gr = 0.0, gi = 0.0;
            for (int k = 0; k < nu; ++k) {
                gr += up[k] * tr[warp][k];
                gi += up[k] * ti[warp][k];
            }
            const int et = a.tmap[e];
            if (et < 0) continue;
            const size_t o = ((16 * (size_t)et + 4 * r + warp) * a.n_z + iz) * 2;
            a.G[o] = gr;
            a.G[o + 1] = gi;
        }
        __syncwarp();
    }
}

void green_columns_eval(const DensityArgs& a, cudaStream_t st) {
    const int n = a.atom_end - a.atom_begin;
    if (n > 0 && a.n_z > 0) k_green<<<n, 128, 0, st>>>(a);
}

}  // namespace elses
