// a2: Slater-Koster H and S on the BSR pattern; a10: forces from rho and rhoE.
//
// H and S are the sparse real-symmetric LCAO matrices of Eq. 1, built locally for the pattern
// (every node of the paper's code computes the elements it needs redundantly instead of
// communicating them). Forces: the gradient of the free energy at fixed electron count is the
// gradient of Omega at fixed mu, with dOmega/dH_ji = rho_ij and dOmega/dS_ji = -rhoE_ij; a block
// (I, J) depends on d = R_J - R_I only, so
//     F_K = sum over blocks e = (K, I) of g_e - g_(I,K),
//     g_e = rho[e] : dH(d_e)/dd - rhoE[e] : dS(d_e)/dd,
// which is summed per atom in a fixed order (no atomics).
#include "internal.h"

namespace elses {

__global__ void k_row_of(int n, const int* __restrict__ row_ptr, int* __restrict__ row_of) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) row_of[e] = i;
}

__device__ __forceinline__ int find_in_row(const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                                           int row, int col) {
    int lo = row_ptr[row], hi = row_ptr[row + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = col_idx[mid];
        if (v == col) return mid;
        if (v < col) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__global__ void k_sk_build(const double* __restrict__ pos, double Lx, double Ly, double Lz, SKDev sk,
                           const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                           const int* __restrict__ row_of, int nnzb, int* __restrict__ tmap,
                           double* __restrict__ H, double* __restrict__ S, double* __restrict__ skr) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnzb) return;
    const int I = row_of[e], J = col_idx[e];
    tmap[e] = find_in_row(row_ptr, col_idx, J, I);
    double hb[16], sb[16];
    if (I == J) {
#pragma unroll
        for (int q = 0; q < 16; ++q) { hb[q] = 0.0; sb[q] = 0.0; }
        hb[0] = sk.Es; hb[5] = sk.Ep; hb[10] = sk.Ep; hb[15] = sk.Ep;
        sb[0] = 1.0; sb[5] = 1.0; sb[10] = 1.0; sb[15] = 1.0;
        // on-site record: u = 0 reduces the two-centre product to diag(ss, pi, pi, pi)
        double* q = skr + 12 * (size_t)e;
        q[0] = 0.0; q[1] = 0.0; q[2] = 0.0; q[3] = 0.0;
        q[4] = sk.Es; q[5] = 0.0; q[6] = sk.Ep; q[7] = 0.0;
        q[8] = 1.0; q[9] = 0.0; q[10] = 1.0; q[11] = 0.0;
    } else {
        const double dx = min_image(pos[3 * J] - pos[3 * I], Lx);
        const double dy = min_image(pos[3 * J + 1] - pos[3 * I + 1], Ly);
        const double dz = min_image(pos[3 * J + 2] - pos[3 * I + 2], Lz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double u[3] = {dx / r, dy / r, dz / r};
        double V[4], dV[4], W[4];
        sk_radial(sk, sk.V0, sk.qH, r, V, dV);
        sk_block(u, V, hb);
        sk_radial(sk, sk.S0, sk.qS, r, W, dV);
        sk_block(u, W, sb);
        // two-centre record for the structured block products: u, then (ss, sp, pp_pi,
        // pp_sigma - pp_pi) of H and of S
        double* q = skr + 12 * (size_t)e;
        q[0] = u[0]; q[1] = u[1]; q[2] = u[2]; q[3] = 0.0;
        q[4] = V[0]; q[5] = V[1]; q[6] = V[3]; q[7] = V[2] - V[3];
        q[8] = W[0]; q[9] = W[1]; q[10] = W[3]; q[11] = W[2] - W[3];
    }
    double2* H2 = reinterpret_cast<double2*>(H + 16 * (size_t)e);
    double2* S2 = reinterpret_cast<double2*>(S + 16 * (size_t)e);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        H2[q] = make_double2(hb[2 * q], hb[2 * q + 1]);
        S2[q] = make_double2(sb[2 * q], sb[2 * q + 1]);
    }
}

void sk_build(const double* pos, int n, const double L[3], const SKDev& sk, const int* row_ptr,
              const int* col_idx, int nnzb, int* row_of, int* tmap, double* H, double* S,
              double* skr, cudaStream_t st) {
    const int T = 256;
    k_row_of<<<(n + T - 1) / T, T, 0, st>>>(n, row_ptr, row_of);
    k_sk_build<<<(nnzb + T - 1) / T, T, 0, st>>>(pos, L[0], L[1], L[2], sk, row_ptr, col_idx, row_of,
                                                 nnzb, tmap, H, S, skr);
}

// g_e for every off-diagonal block (zero on the diagonal).
__global__ void k_force_blocks(const double* __restrict__ pos, double Lx, double Ly, double Lz, SKDev sk,
                               const int* __restrict__ col_idx, const int* __restrict__ row_of, int nnzb,
                               const double* __restrict__ rho, const double* __restrict__ rhoE,
                               double* __restrict__ g_block) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnzb) return;
    const int I = row_of[e], J = col_idx[e];
    double g[3] = {0.0, 0.0, 0.0};
    if (I != J) {
        const double dx = min_image(pos[3 * J] - pos[3 * I], Lx);
        const double dy = min_image(pos[3 * J + 1] - pos[3 * I + 1], Ly);
        const double dz = min_image(pos[3 * J + 2] - pos[3 * I + 2], Lz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double u[3] = {dx / r, dy / r, dz / r};
        double R[16], V[4], dV[4], gh[3], gs[3];
#pragma unroll
        for (int q = 0; q < 16; ++q) R[q] = rho[16 * (size_t)e + q];
        sk_radial(sk, sk.V0, sk.qH, r, V, dV);
        sk_block_grad_dot(u, r, V, dV, R, gh);
#pragma unroll
        for (int q = 0; q < 16; ++q) R[q] = rhoE[16 * (size_t)e + q];
        sk_radial(sk, sk.S0, sk.qS, r, V, dV);
        sk_block_grad_dot(u, r, V, dV, R, gs);
#pragma unroll
        for (int m = 0; m < 3; ++m) g[m] = gh[m] - gs[m];
    }
    g_block[3 * (size_t)e] = g[0];
    g_block[3 * (size_t)e + 1] = g[1];
    g_block[3 * (size_t)e + 2] = g[2];
}

__global__ void k_force_atoms(int n, const int* __restrict__ row_ptr, const int* __restrict__ tmap,
                              const double* __restrict__ g_block, double* __restrict__ F) {
    int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= n) return;
    double f[3] = {0.0, 0.0, 0.0};
    for (int e = row_ptr[K]; e < row_ptr[K + 1]; ++e) {
        const int t = tmap[e];
        if (t < 0) continue;   // the pattern is symmetric by construction; never taken
#pragma unroll
        for (int m = 0; m < 3; ++m) f[m] += g_block[3 * (size_t)e + m] - g_block[3 * (size_t)t + m];
    }
    F[3 * K] = f[0];
    F[3 * K + 1] = f[1];
    F[3 * K + 2] = f[2];
}

void forces(const double* pos, int n, const double L[3], const SKDev& sk, const int* row_ptr,
            const int* col_idx, const int* row_of, const int* tmap, int nnzb, const double* rho,
            const double* rhoE, double* g_block, double* F, cudaStream_t st) {
    const int T = 256;
    k_force_blocks<<<(nnzb + T - 1) / T, T, 0, st>>>(pos, L[0], L[1], L[2], sk, col_idx, row_of, nnzb,
                                                     rho, rhoE, g_block);
    k_force_atoms<<<(n + T - 1) / T, T, 0, st>>>(n, row_ptr, tmap, g_block, F);
}

// (pi)COHP integrals of Eqs. 4-8 per block e = (I, J): B = sum_ab H[e][a][b] rho[e][a][b] (H is
// symmetric, so H_(J,b);(I,a) = H[e][a][b]); the pi part takes only the V_pp_pi (delta_ik - u_i u_k)
// term of the p-p block, sigma = B - pi off-site; on-site blocks carry no split.
__global__ void k_icohp(const double* __restrict__ pos, double Lx, double Ly, double Lz, SKDev sk,
                        const int* __restrict__ col_idx, const int* __restrict__ row_of, int nnzb,
                        const double* __restrict__ H, const double* __restrict__ rho,
                        double* __restrict__ B, double* __restrict__ Bsig, double* __restrict__ Bpi) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnzb) return;
    double b = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) b = fma(H[16 * (size_t)e + q], rho[16 * (size_t)e + q], b);
    B[e] = b;
    if (!Bsig && !Bpi) return;
    const int I = row_of[e], J = col_idx[e];
    double bpi = 0.0;
    if (I != J) {
        const double dx = min_image(pos[3 * J] - pos[3 * I], Lx);
        const double dy = min_image(pos[3 * J + 1] - pos[3 * I + 1], Ly);
        const double dz = min_image(pos[3 * J + 2] - pos[3 * I + 2], Lz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double u[3] = {dx / r, dy / r, dz / r};
        double V[4], dV[4];
        sk_radial(sk, sk.V0, sk.qH, r, V, dV);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                bpi = fma(V[3] * ((i == k ? 1.0 : 0.0) - u[i] * u[k]), rho[16 * (size_t)e + 4 * (1 + i) + 1 + k], bpi);
    }
    if (Bpi) Bpi[e] = bpi;
    if (Bsig) Bsig[e] = (I != J) ? b - bpi : 0.0;
}

// Eq. 4 at complex energies: C_e(z) = -(1/pi) Im sum_ab H_e[a][b] G_e[a][b](z) for block e = (I, J)
// (H symmetric: H_(J,b);(I,a) = H_e[a][b]) and its pi part from the V_pp_pi term of the p-p block,
// for the n_zc energies of a chunk of G ([e*16 + q][n_zc][2]); outputs [e][n_z] from column iz0.
__global__ void k_cohp(const double* __restrict__ pos, double Lx, double Ly, double Lz, SKDev sk,
                       const int* __restrict__ col_idx, const int* __restrict__ row_of, int nnzb,
                       const double* __restrict__ H, const double* __restrict__ G, int n_zc, int iz0, int n_z,
                       double* __restrict__ C, double* __restrict__ Csig, double* __restrict__ Cpi) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nnzb * n_zc) return;
    const int e = (int)(t / n_zc), iz = (int)(t - (size_t)e * n_zc);
    const double* g = G + (16 * (size_t)e * n_zc + iz) * 2 + 1;    // Im G_e[q], stride 2 n_zc
    const size_t st = 2 * (size_t)n_zc;
    double c = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) c = fma(H[16 * (size_t)e + q], g[q * st], c);
    const double inv_pi = 0.31830988618379067154;
    const size_t o = (size_t)e * n_z + iz0 + iz;
    if (C) C[o] = -inv_pi * c;
    if (!Csig && !Cpi) return;
    const int I = row_of[e], J = col_idx[e];
    double cpi = 0.0;
    if (I != J) {
        const double dx = min_image(pos[3 * J] - pos[3 * I], Lx);
        const double dy = min_image(pos[3 * J + 1] - pos[3 * I + 1], Ly);
        const double dz = min_image(pos[3 * J + 2] - pos[3 * I + 2], Lz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double u[3] = {dx / r, dy / r, dz / r};
        double V[4], dV[4];
        sk_radial(sk, sk.V0, sk.qH, r, V, dV);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                cpi = fma(V[3] * ((i == k ? 1.0 : 0.0) - u[i] * u[k]), g[(4 * (1 + i) + 1 + k) * st], cpi);
    }
    if (Cpi) Cpi[o] = -inv_pi * cpi;
    if (Csig) Csig[o] = (I != J) ? -inv_pi * (c - cpi) : 0.0;
}

void icohp(const double* pos, const double L[3], const SKDev& sk, const int* col_idx, const int* row_of,
           int nnzb, const double* H, const double* rho, double* B, double* Bsig, double* Bpi, cudaStream_t st) {
    const int T = 256;
    k_icohp<<<(nnzb + T - 1) / T, T, 0, st>>>(pos, L[0], L[1], L[2], sk, col_idx, row_of, nnzb, H, rho, B,
                                              Bsig, Bpi);
}

void cohp_spectrum(const double* pos, const double L[3], const SKDev& sk, const int* col_idx, const int* row_of,
                   int nnzb, const double* H, const double* G, int n_zc, int iz0, int n_z, double* C,
                   double* Csig, double* Cpi, cudaStream_t st) {
    const int T = 256;
    const size_t n = (size_t)nnzb * n_zc;
    k_cohp<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(pos, L[0], L[1], L[2], sk, col_idx, row_of, nnzb, H, G,
                                                      n_zc, iz0, n_z, C, Csig, Cpi);
}

}  // namespace elses
