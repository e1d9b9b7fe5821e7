// a8: density-matrix columns on the pattern; G_ij(z) on the pattern for given z.
//
// Eq. 2: rho_ij = -(1/pi) Int f(e - mu) Im G_ij(e + i0) de. With G_ij(z) = sum_k Z_ik c_k /
// (z - e_k) the integral is taken by residues (Im 1/(e + i0 - e_k) = -pi delta(e - e_k)):
//     rho_ij  = 2 sum_k f(e_k - mu) Z_ik c_k          (2: spin)
//     rhoE_ij = 2 sum_k f(e_k - mu) e_k Z_ik c_k
// for the pattern rows i of column j (atoms within r_cut of J), with Z = U V. Computed as
// t = V (2 f c) (nu x nu) followed by rho_P = U_P t, which needs no Z. Where V is not formed, t
// comes from the eigen-factors (k_eig_weights).
//
// One CTA per atom J, one warp per column; column j = 4J + b writes rho[(I, J)][a][b] through
// the transpose map of the pattern (each element is written exactly once).
#include "internal.h"

namespace elses {

__global__ void __launch_bounds__(128) k_density(const DensityArgs a) {
    __shared__ double wc[4][kMaxNu], wec[4][kMaxNu], t[4][kMaxNu], tE[4][kMaxNu];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int J = a.atom_begin + blockIdx.x;
    if (J >= a.atom_end) return;
    const int j = 4 * J + warp;
    const int nm = a.nu_max;
    const int nu = a.nu_eff[j];
    if (a.T) {   // t and t_E from the eigen-factors (k_eig_weights)
        const double* u = a.T + (size_t)(j - a.v_col0) * 2 * nm;
        for (int n = lane; n < nu; n += 32) {
            t[warp][n] = u[n];
            tE[warp][n] = u[nm + n];
        }
    } else {
        const double mu = a.mu_dev ? *a.mu_dev : a.mu;
        for (int k = lane; k < nu; k += 32) {
            const double e = a.eps[(size_t)j * nm + k];
            const double f2 = 2.0 * fermi((e - mu) / a.kT) * a.c[(size_t)j * nm + k];
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
