// Shared device helpers of the GB300 per-column Krylov library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "elses.h"

namespace elses {

// Device-side error flags (OR-ed into one status word; mapped to ELSES_ERR_* on the host).
enum : int {
    DEV_NOT_SPD = 1,
    DEV_NONFINITE = 2,
    DEV_CAPACITY = 4,
    DEV_TIMEOUT = 8,
    DEV_BREAKDOWN = 16,   // informational: nu_eff < nu for some column
    DEV_NO_BRACKET = 32,
    DEV_ARG = 64,
};

constexpr int kMaxNu = 64;          // Krylov dimension limit (registers / shared arrays)
constexpr int kWarpsPerAtom = 4;    // one warp per orbital column of an atom

// Raises a kernel's dynamic shared-memory limit to at least `bytes` and never lowers it: the limit
// is a property of the function, shared by every system on the device, and after the first
// launches no attribute call stays on the launch path (where it could order launches that are
// meant to overlap).
template <typename Kernel>
inline void smem_at_least(Kernel kernel, size_t bytes) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes >= bytes) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    // the whole L1 / shared split as shared memory: launches of the same kernel with different
    // footprints (the cluster size classes) then share one SM configuration and can co-reside
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// For kernels that stream per-thread data through L1 (one thread per column reading its own
// lists): the shared memory of the CTAs a grid of `grid` CTAs puts on an SM, at most
// `max_ctas` of them where it is set, the rest of the unified L1 / shared storage left to L1.
// By default the driver sizes shared memory for the kernel's maximum occupancy, which leaves L1
// too small for these streams; a grid of many waves would do the same without the cap.
template <typename Kernel>
inline void carveout_for(Kernel kernel, size_t bytes, int grid, int max_ctas = 0) {
    int dev = 0, sms = 1, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (smem_sm <= 0 || sms <= 0) return;
    size_t ctas = (size_t)(grid + sms - 1) / sms;
    if (max_ctas > 0) ctas = std::min<size_t>(ctas, (size_t)max_ctas);
    const size_t need = ctas * (bytes + 1024);   // + the per-CTA reservation
    const int pct = (int)std::min<size_t>(100, (need * 100 + smem_sm - 1) / (size_t)smem_sm);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

__device__ __forceinline__ void flag(int* st, int f) { atomicOr(st, f); }

// Fermi-Dirac occupation f = 1 / (1 + exp(x)), x = (e - mu) / kT, without overflow.
__device__ __forceinline__ double fermi(double x) {
    if (x > 0.0) {
        const double t = exp(-x);
        return t / (1.0 + t);
    }
    return 1.0 / (1.0 + exp(x));
}

// Grand-potential weight w(e) = -2 kT ln(1 + exp(-(e - mu)/kT)); dw/de = 2 f.
__device__ __forceinline__ double omega_w(double e, double mu, double kT) {
    const double x = (e - mu) / kT;
    if (x >= 0.0) return -2.0 * kT * log1p(exp(-x));
    return 2.0 * (x * kT) - 2.0 * kT * log1p(exp(x));
}

// Minimum image with one IEEE operation per step, in the fixed order d - L*rint(d/L). No FMA
// contraction: the integer outputs (neighbour lists) must be reproducible bit for bit.
__device__ __forceinline__ double min_image(double d, double L) {
    double q = rint(__ddiv_rn(d, L));
    return __dsub_rn(d, __dmul_rn(L, q));
}

// (dx*dx + dy*dy) + dz*dz with every product and sum rounded separately.
__device__ __forceinline__ double dist2_exact(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Butterfly sum of one double over the 32 lanes of a warp (result in every lane).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of 32 values held by every lane over the 32 lanes, by recursive halving: after the call
// lane l holds in v[0] the warp-wide sum of value l. 31 additions per lane for 32 values.
__device__ __forceinline__ double warp_sum32(double (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            double send = upper ? v[i] : v[i + w];
            double keep = upper ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

// ---------------------------------------------------------------- Slater-Koster (device)
struct SKDev {
    double Es, Ep;
    double V0[4], qH[4], S0[4], qS[4];
    double r0, r_on, r_cut;
};

__device__ __forceinline__ void sk_taper(const SKDev& sk, double r, double& t, double& dt) {
    if (r <= sk.r_on) { t = 1.0; dt = 0.0; return; }
    if (r >= sk.r_cut) { t = 0.0; dt = 0.0; return; }
    const double w = sk.r_cut - sk.r_on;
    const double s = (r - sk.r_on) / w;
    const double s2 = s * s, s3 = s2 * s;
    t = 1.0 + s3 * (-10.0 + s * (15.0 - 6.0 * s));
    dt = s2 * (-30.0 + s * (60.0 - 30.0 * s)) / w;
}

// Radial integrals V_x(r) = V0_x exp(-q_x (r - r0)) t(r) and their r-derivatives.
__device__ __forceinline__ void sk_radial(const SKDev& sk, const double* V0, const double* q,
                                          double r, double V[4], double dV[4]) {
    double t, dt;
    sk_taper(sk, r, t, dt);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const double e = V0[x] * exp(-q[x] * (r - sk.r0));
        V[x] = e * t;
        dV[x] = e * (dt - q[x] * t);
    }
}

// 4x4 block of the pair at d = R_J - R_I from unit vector u and integrals V (row-major).
__device__ __forceinline__ void sk_block(const double u[3], const double V[4], double B[16]) {
    B[0] = V[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        B[1 + i] = u[i] * V[1];
        B[4 * (1 + i)] = -u[i] * V[1];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            B[4 * (1 + i) + 1 + k] = u[i] * u[k] * (V[2] - V[3]) + (i == k ? V[3] : 0.0);
    }
}

// Contraction sum_ab R[a][b] d(block)[a][b]/d(d_m) for m = 0..2 (R row-major 4x4).
__device__ __forceinline__ void sk_block_grad_dot(const double u[3], double r, const double V[4],
                                                  const double dV[4], const double R[16],
                                                  double g[3]) {
    const double inv_r = 1.0 / r;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        double acc = R[0] * dV[0] * u[m];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double dui = ((i == m ? 1.0 : 0.0) - u[i] * u[m]) * inv_r;
            const double sp = dV[1] * u[m] * u[i] + V[1] * dui;
            acc += (R[1 + i] - R[4 * (1 + i)]) * sp;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double duk = ((k == m ? 1.0 : 0.0) - u[k] * u[m]) * inv_r;
                const double pp = (dV[2] - dV[3]) * u[m] * u[i] * u[k] +
                                  (i == k ? dV[3] * u[m] : 0.0) +
                                  (V[2] - V[3]) * (dui * u[k] + u[i] * duk);
                acc += R[4 * (1 + i) + 1 + k] * pp;
            }
        }
        g[m] = acc;
    }
}

}  // namespace elses
