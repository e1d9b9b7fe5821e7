// a5 + a6: projected generalized eigenproblem H' v = e S' v per column, and its spectra.
//
// Eq. 1 is solved instead of the generalized eigenvalue equation H y = e S y of the whole
// system; on the nu-dimensional Krylov space of a column that equation is small and is solved
// exactly:  S' = L L^T (Cholesky),  A = L^-1 H' L^-T,  A = Q diag(e) Q^T,  V = L^-T Q.
// The Green's-function column then has poles e_k and residues Z_ik c_k with Z = U V and
// c = V^T U^T e_j; kept per column are (e, c, d = V^T (SU)_j, g = V^T (HU)_j) and V.
//
// GB300 form. On this part the FP64 pipe charges a whole warp instruction whatever the number
// of active lanes, so every FP64 instruction must carry work on all lanes:
//   k_eig_reduce   one warp per column, matrices in shared memory: Cholesky, the reduction
//                  A = L^-1 H' L^-T and the Householder reduction of A to tridiagonal form T
//                  (lanes over rows / columns); the three vectors z = L^-1 (U, SU, HU)_j are
//                  reflected along, y = Q_H^T z.
//   k_eig_chase    one thread per column: implicit-shift QR sweeps on T (Wilkinson shift, Givens
//                  bulge chase) -- the sequential part; the rotations are recorded.
//   k_eig_spectra  one thread per (column, vector): the rotations replayed on y give
//                  c, d, g = Q^T z.
//   k_eig_vectors  one warp per column, only where V itself is needed (G(z), the adjoint, or
//                  batches that overwrite the factors): Q_H from the reflectors, the rotations
//                  applied to its columns, V = L^-T Q; when V is formed with the columns, the
//                  spectra c, d, g = Q^T z too (instead of k_eig_spectra).
//   k_eig_weights  one thread per (column, vector): the density needs V only applied to two
//                  vectors, t = V w = L^-T Q_H (R_1^T .. R_n^T w), taken from the factors.
//   k_eig_archive  several batches: each batch's factors into the archive of every column
//                  (reflectors and L packed, rotations in a shared pool), so that the density
//                  reads them after the last batch instead of V formed per batch; columns the
//                  pool cannot hold get V (k_eig_vectors_listed).
#include <algorithm>

#include "internal.h"

namespace elses {

__host__ __device__ size_t eig_tri_doubles(int nm) { return 5 * (size_t)nm; }        // D, E, y (3 vectors)
// reflector k in row k (entries i > k, tau_k at k), then L row-major
__host__ __device__ size_t eig_fac_doubles(int nm) { return 2 * (size_t)nm * nm; }
__host__ __device__ size_t eig_rot_cap(int nm) { return 2 * (size_t)nm * nm + 64; }  // Givens rotations per column
__host__ __device__ size_t eig_arch_fac_doubles(int nm) { return (size_t)nm * (nm + 1); }  // both triangles packed
constexpr int kRotStage = 128;   // rotations staged in shared memory at a time (k_eig_vectors)
constexpr int kChaseThreads = 64;  // columns per CTA of k_eig_chase
// CTAs per SM that the shared memory of the rotation-replay kernels (k_eig_spectra,
// k_eig_weights) is sized for on grids of many waves: each thread streams its own rotation
// list, and with more CTAs the L1 left over no longer holds the warps' streams
constexpr int kStreamCtas = 8;

// The lower-triangle pairs (i, m), lo <= m <= i < hi, in row-major order, 32 at a time from
// `lane`: f(i, m) for each pair the lane owns. Trailing-block updates spread this way keep all
// lanes busy (lanes over rows leave most of them idle as the block shrinks), and on this part an
// FP64 warp instruction costs the same whatever the number of active lanes.
template <typename F>
__device__ __forceinline__ void lower_pairs(int lo, int hi, int lane, F f) {
    const int n = hi - lo;
    int r = 0, q = lane;                       // row r = i - lo holds the r + 1 pairs q = 0 .. r
    while (r < n && q > r) { q -= r + 1; ++r; }
    while (r < n) {
        f(lo + r, lo + q);
        q += 32;
        while (r < n && q > r) { q -= r + 1; ++r; }
    }
}

// packed upper storage: element (i, k), i <= k, at i + k (k + 1) / 2
__device__ __forceinline__ double packed(const double* P, int i, int k) {
    return i <= k ? P[i + k * (k + 1) / 2] : P[k + i * (i + 1) / 2];
}

// ----------------------------------------------------------------------------- k_eig_reduce
__global__ void __launch_bounds__(64) k_eig_reduce(const EigArgs a) {
    extern __shared__ __align__(16) double sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + wib;
    if (c >= a.ncols) return;
    const int nm = a.nu_max, ld = nm + 1;
    double* A = sm + (size_t)wib * ((2 * nm + 3) * ld + 2 * nm + 3);
    double* L = A + (nm + 3) * ld;  // A: the matrix, then the three vectors as rows nu .. nu + 2
    double* inv = L + nm * ld;     // 1 / L_ii
    double* P = inv + nm;          // Householder work vector (nm + 3)
    double* yv = a.tri + (size_t)c * eig_tri_doubles(nm);   // D, E, yc, yd, yg (global)
    const int j = a.col0 + c;
    const int nu = a.nu_eff[j];
    const int PK = nm * (nm + 1) / 2;
    const double* Hp = a.Hp + (size_t)c * PK;
    const double* Sp = a.Sp + (size_t)c * PK;

    for (int q = lane; q < nu * nu; q += 32) {
        const int i = q / nu, k = q % nu;
        A[i * ld + k] = packed(Hp, i, k);
        L[i * ld + k] = packed(Sp, i, k);
    }
    __syncwarp();
    // Cholesky S' = L L^T (right-looking, lanes over rows of the trailing block)
    bool spd = true;
    for (int k = 0; k < nu; ++k) {
        const double dk = L[k * ld + k];
        if (!(dk > 0.0)) { spd = false; break; }
        const double ik = rsqrt(dk), lkk = dk * ik;   // one reciprocal square root, no division
        __syncwarp();
        for (int i = k + 1 + lane; i < nu; i += 32) L[i * ld + k] *= ik;
        if (lane == 0) { L[k * ld + k] = lkk; inv[k] = ik; }
        __syncwarp();
        lower_pairs(k + 1, nu, lane, [&](int i, int m) {
            L[i * ld + m] = fma(-L[i * ld + k], L[m * ld + k], L[i * ld + m]);
        });
        __syncwarp();
    }
    if (!spd) {
        if (lane == 0) flag(a.status, DEV_NOT_SPD);
        for (int q = lane; q < 5 * nm; q += 32) yv[q] = 0.0;
        return;
    }
    // X = L^-1 H' in place (lanes over columns n), then A = X L^-T in place (lanes over rows i)
    for (int n = lane; n < nu; n += 32)
        for (int i = 0; i < nu; ++i) {
            double s = A[i * ld + n];
            for (int m = 0; m < i; ++m) s = fma(-L[i * ld + m], A[m * ld + n], s);
            A[i * ld + n] = s * inv[i];
        }
    __syncwarp();
    for (int i = lane; i < nu; i += 32)
        for (int n = 0; n < nu; ++n) {
            double s = A[i * ld + n];
            for (int m = 0; m < n; ++m) s = fma(-A[i * ld + m], L[n * ld + m], s);
            A[i * ld + n] = s * inv[n];
        }
    __syncwarp();
    for (int i = lane; i < nu; i += 32)
        for (int k = 0; k < i; ++k) {
            const double v = 0.5 * (A[i * ld + k] + A[k * ld + i]);
            A[i * ld + k] = v;
            A[k * ld + i] = v;
        }
    __syncwarp();
    // the three vectors z = L^-1 (U, SU, HU)_j into rows nu .. nu + 2 of A: a column sweep with
    // lanes over rows (rows lane and lane + 32), row m final at step m
    {
        const double* src[3] = {a.urow + (size_t)c * nm, a.surow + (size_t)c * nm, a.hurow + (size_t)c * nm};
        double z0[3], z1[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            z0[q] = lane < nu ? src[q][lane] : 0.0;
            z1[q] = lane + 32 < nu ? src[q][lane + 32] : 0.0;
        }
        for (int m = 0; m < nu; ++m) {
            const int owner = m & 31;
            const bool upper = m >= 32;
            const double im = inv[m];
            double y[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) y[q] = __shfl_sync(0xffffffffu, (upper ? z1[q] : z0[q]) * im, owner);
            if (lane == owner) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (upper) z1[q] = y[q]; else z0[q] = y[q];
                }
            }
            if (lane > m && lane < nu) {
                const double l = L[lane * ld + m];
#pragma unroll
                for (int q = 0; q < 3; ++q) z0[q] = fma(-l, y[q], z0[q]);
            }
            if (lane + 32 > m && lane + 32 < nu) {
                const double l = L[(lane + 32) * ld + m];
#pragma unroll
                for (int q = 0; q < 3; ++q) z1[q] = fma(-l, y[q], z1[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (lane < nu) A[(nu + q) * ld + lane] = z0[q];
            if (lane + 32 < nu) A[(nu + q) * ld + lane + 32] = z1[q];
        }
    }
    __syncwarp();
    // Householder reduction: reflector k stored in column k below the diagonal, tau_k kept; the
    // vector rows are reflected along (y = Q_H^T z). The trailing block is kept in its lower
    // triangle only (read symmetrically).
    double* E = yv + nm;
    for (int k = 0; k + 2 < nu; ++k) {
        double part = 0.0;
        for (int i = k + 1 + lane; i < nu; i += 32) part = fma(A[i * ld + k], A[i * ld + k], part);
        const double sigma = warp_sum(part);
        const double x0 = A[(k + 1) * ld + k];
        __syncwarp();
        if (sigma == 0.0) {
            if (lane == 0) { E[k] = 0.0; P[k] = 0.0; }
            continue;
        }
        const double alpha = -copysign(sqrt(sigma), x0);
        const double tau = 1.0 / (alpha * (alpha - x0));
        if (lane == 0) A[(k + 1) * ld + k] = x0 - alpha;
        __syncwarp();
        // p = tau A v (rows i > k); the same sweep gives t_q = tau v^T y_q for the vector rows,
        // in lanes the matrix rows leave idle
        double kp = 0.0;
        for (int i = k + 1 + lane; i < nu + 3; i += 32) {
            double s = 0.0;
            for (int m = k + 1; m < nu; ++m) s = fma(m <= i ? A[i * ld + m] : A[m * ld + i], A[m * ld + k], s);
            s *= tau;
            P[i] = s;
            if (i < nu) kp = fma(A[i * ld + k], s, kp);
        }
        const double K = 0.5 * tau * warp_sum(kp);
        __syncwarp();
        for (int i = k + 1 + lane; i < nu; i += 32) P[i] = fma(-K, A[i * ld + k], P[i]);
        __syncwarp();
        lower_pairs(k + 1, nu, lane, [&](int i, int m) {
            A[i * ld + m] = fma(-A[i * ld + k], P[m], fma(-P[i], A[m * ld + k], A[i * ld + m]));
        });
        for (int m = k + 1 + lane; m < nu; m += 32) {   // y_q -= t_q v
            const double vm = A[m * ld + k];
#pragma unroll
            for (int q = 0; q < 3; ++q) A[(nu + q) * ld + m] = fma(-P[nu + q], vm, A[(nu + q) * ld + m]);
        }
        __syncwarp();
        if (lane == 0) { E[k] = alpha; P[k] = tau; }   // P[k] keeps tau_k (P[i > k] reused later)
        __syncwarp();
    }
    // tridiagonal T: D, E
    double* D = yv;
    for (int i = lane; i < nu; i += 32) D[i] = A[i * ld + i];
    if (lane == 0 && nu >= 2) E[nu - 2] = A[(nu - 1) * ld + (nu - 2)];
    if (lane == 0 && nu >= 2) {
        // the last two reflector slots are unused: mark them
        P[nu - 2] = 0.0;
        P[nu - 1] = 0.0;
    }
    __syncwarp();
    // the three vectors y = Q_H^T z
    for (int q = lane; q < 3 * nu; q += 32) {
        const int v = q / nu, m = q % nu;
        yv[(2 + v) * nm + m] = A[(nu + v) * ld + m];
    }
    __syncwarp();
    // factors: reflector k as row k of the first matrix (its entries i > k, tau_k at k), L
    double* F = a.fac + (size_t)c * eig_fac_doubles(nm);
    for (int q = lane; q < nu * nu; q += 32) {
        const int k = q / nu, i = q % nu;
        F[k * nm + i] = (i == k) ? P[k] : A[i * ld + k];
        F[nm * nm + k * nm + i] = L[k * ld + i];
    }
}

// ----------------------------------------------------------------------------- k_eig_chase
// A thread's array in shared memory, element i at p[i * kChaseThreads] (conflict-free: the
// threads of a warp touch consecutive words for equal i).
template <int kStride>
struct Strided {
    double* p;
    __device__ __forceinline__ double& operator[](int i) const { return p[(size_t)i * kStride]; }
};
using ThreadArray = Strided<kChaseThreads>;

__global__ void __launch_bounds__(kChaseThreads) k_eig_chase(const EigArgs a) {
    extern __shared__ double csm[];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.ncols) return;
    const int nm = a.nu_max;
    const int j = a.col0 + c;
    const int nu = a.nu_eff[j];
    // the thread's tridiagonal moves to shared memory for the chase: the latency of every access
    // stays that of shared memory however many columns are in flight
    double* base = csm + threadIdx.x;
    const ThreadArray D{base}, E{base + (size_t)nm * kChaseThreads};
    {
        const double* t = a.tri + (size_t)c * eig_tri_doubles(nm);
        for (int k = 0; k < nu; ++k) {
            D[k] = t[k];
            if (k + 1 < nu) E[k] = t[nm + k];
        }
    }
    double* rc = a.rot_c + (size_t)c * eig_rot_cap(nm);
    double* rs = a.rot_s + (size_t)c * eig_rot_cap(nm);
    unsigned char* rk = a.rot_k + (size_t)c * eig_rot_cap(nm);
    const size_t cap = eig_rot_cap(nm);
    size_t nrot = 0;
    bool ok = true;
    const double eps = 2.220446049250313e-16;
    int hi = nu - 1, sweeps = 0;
    const int max_sweeps = a.max_sweeps > 0 ? a.max_sweeps : 30 * nu;
    // each pass deflates every negligible trailing off-diagonal entry, then makes one sweep:
    // the columns of a warp then reach their sweeps together (a column that deflated would
    // otherwise sit out the other lanes' sweep), in the same order of operations per column.
    // A column without a space (nu = 0, flagged by the Krylov build) has nothing to chase.
    while (ok && hi > 0) {
        while (hi > 0 && fabs(E[hi - 1]) <= eps * (fabs(D[hi - 1]) + fabs(D[hi]))) {
            E[hi - 1] = 0.0;
            --hi;
        }
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && fabs(E[lo - 1]) > eps * (fabs(D[lo - 1]) + fabs(D[lo]))) --lo;
        if (lo > 0) E[lo - 1] = 0.0;
        if (++sweeps > max_sweeps || nrot + (hi - lo) > cap) {
            ok = false;
            break;
        }
        const double delta = 0.5 * (D[hi - 1] - D[hi]);
        const double b2 = E[hi - 1] * E[hi - 1];
        const double den = delta + copysign(sqrt(delta * delta + b2), delta);
        const double mu = D[hi] - (den != 0.0 ? b2 / den : 0.0);
        double x = D[lo] - mu, z = E[lo];
        for (int k = lo; k < hi; ++k) {
            // c = x / r, s = z / r, r = |(x, z)| from one reciprocal square root
            const double rr = fma(x, x, z * z);
            double cr = 1.0, sr = 0.0, r = 0.0;
            if (rr > 0.0) {
                const double ir = rsqrt(rr);
                cr = x * ir;
                sr = z * ir;
                r = rr * ir;
            }
            if (k > lo) E[k - 1] = r;
            const double ak = D[k], ak1 = D[k + 1], b = E[k];
            const double cc = cr * cr, ss = sr * sr, cs = cr * sr;
            D[k] = cc * ak + 2.0 * cs * b + ss * ak1;
            D[k + 1] = ss * ak - 2.0 * cs * b + cc * ak1;
            E[k] = cs * (ak1 - ak) + (cc - ss) * b;
            if (k + 1 < hi) {
                const double bn = E[k + 1];
                z = sr * bn;
                E[k + 1] = cr * bn;
                x = E[k];
            }
            rc[nrot] = cr;
            rs[nrot] = sr;
            rk[nrot] = (unsigned char)k;
            ++nrot;
        }
    }
    if (!ok) flag(a.status, DEV_TIMEOUT);
    a.rot_n[c] = ok ? (int)nrot : 0;
    // ascending order; perm[out] = index into the unsorted arrays
    int* perm = a.perm + (size_t)c * nm;
    for (int k = 0; k < nu; ++k) perm[k] = k;
    for (int k = 0; k + 1 < nu; ++k) {
        int m = k;
        for (int q = k + 1; q < nu; ++q)
            if (D[perm[q]] < D[perm[m]]) m = q;
        const int tmp = perm[k]; perm[k] = perm[m]; perm[m] = tmp;
    }
    for (int k = 0; k < nm; ++k) a.eps[(size_t)j * nm + k] = (k < nu && ok) ? D[perm[k]] : 0.0;
}

// ----------------------------------------------------------------------------- k_eig_spectra
// The recorded rotations of a column, read in order (forward) or backwards, from its own lists
// (a thread's consecutive reads share cache sectors).
struct RotList {
    const double* c;
    const double* s;
    const unsigned char* k;
    int n;
    __device__ RotList(const EigArgs& a, int col) {
        const size_t o = (size_t)col * eig_rot_cap(a.nu_max);
        c = a.rot_c + o;
        s = a.rot_s + o;
        k = a.rot_k + o;
        n = a.rot_n[col];
    }
};

// Q = Q_H R_1^T .. R_n^T, so Q^T z = R_n .. R_1 y: each recorded rotation, in order, turns
// (y_k, y_k+1) into (c y_k + s y_k+1, c y_k+1 - s y_k). A CTA takes 32 columns and one warp per
// vector (c, d, g): three times the warps of a thread per column for the same instructions, and
// the three threads of a column read its rotation list together. Written in ascending order of
// the poles (zero past nu).
constexpr int kSpecThreads = 96;
__global__ void __launch_bounds__(kSpecThreads) k_eig_spectra(const EigArgs a) {
    extern __shared__ double csm[];
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    if (c >= a.ncols) return;
    const int nm = a.nu_max;
    const int j = a.col0 + c;
    const int nu = a.nu_eff[j];
    const Strided<kSpecThreads> Y{csm + threadIdx.x};
    const double* y = a.tri + (size_t)c * eig_tri_doubles(nm) + (2 + q) * (size_t)nm;
    for (int k = 0; k < nu; ++k) Y[k] = y[k];
    const RotList R(a, c);
    int r = 0;   // the loads of four rotations issued before the four are applied
    for (; r + 3 < R.n; r += 4) {
        double cq[4], sq[4];
        int kq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cq[q] = __ldg(R.c + r + q);
            sq[q] = __ldg(R.s + r + q);
            kq[q] = __ldg(R.k + r + q);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = kq[q];
            const double p = Y[k], w = Y[k + 1];
            Y[k] = fma(cq[q], p, sq[q] * w);
            Y[k + 1] = fma(cq[q], w, -sq[q] * p);
        }
    }
    for (; r < R.n; ++r) {
        const double cr = __ldg(R.c + r), sr = __ldg(R.s + r);
        const int k = __ldg(R.k + r);
        const double p = Y[k], w = Y[k + 1];
        Y[k] = fma(cr, p, sr * w);
        Y[k + 1] = fma(cr, w, -sr * p);
    }
    const int* perm = a.perm + (size_t)c * nm;
    double* out = (q == 0 ? a.c : q == 1 ? a.d : a.g) + (size_t)j * nm;
    for (int k = 0; k < nm; ++k) out[k] = k < nu ? Y[perm[k]] : 0.0;
}

// ----------------------------------------------------------------------------- factor sources
// Where a column's factors are read. The batch buffers (batch column c): reflector k in row k of
// an nm x nm matrix (entries i > k, tau_k at k), L row-major after it, the rotations at
// c * rot_cap. The archive (global column j): the reflectors' upper triangle and L's lower
// triangle packed row by row, the rotations in the pool from off[j].
struct FactorSrc {
    const double* F;          // reflector k, entry i >= k: F[rrow(k) + i]
    const double* Lf;         // L row i, entry l <= i: Lf[lrow(i) + l]
    const int* perm;
    const double* rc;
    const double* rs;
    const unsigned char* rk;
    int nrot;
    int nm;
    bool packed;
    __device__ __forceinline__ long long rrow(int k) const {
        return packed ? (long long)k * nm - (long long)k * (k - 1) / 2 - k : (long long)k * nm;
    }
    __device__ __forceinline__ long long lrow(int i) const {
        return packed ? (long long)i * (i + 1) / 2 : (long long)i * nm;
    }
};

__device__ __forceinline__ FactorSrc batch_factors(const EigArgs& a, int c) {
    const int nm = a.nu_max;
    const size_t o = (size_t)c * eig_rot_cap(nm);
    const double* F = a.fac + (size_t)c * eig_fac_doubles(nm);
    return {F, F + (size_t)nm * nm, a.perm + (size_t)c * nm, a.rot_c + o, a.rot_s + o, a.rot_k + o,
            a.rot_n[c], nm, false};
}

// only for a column the archive holds (n[j] >= 0)
__device__ __forceinline__ FactorSrc archived_factors(const EigArgs& a, int j) {
    const int nm = a.nu_max;
    const unsigned long long o = a.ar.off[j];
    const double* F = a.ar.fac + (size_t)j * eig_arch_fac_doubles(nm);
    return {F, F + (size_t)nm * (nm + 1) / 2, a.ar.perm + (size_t)j * nm, a.ar.rot_c + o, a.ar.rot_s + o,
            a.ar.rot_k + o, a.ar.n[j], nm, true};
}

// ----------------------------------------------------------------------------- k_eig_vectors
// spectra: also write c, d, g = Q^T z in pole order (the batches that form V get them here instead
// of from k_eig_spectra): z = Q_H y is taken with Q_H once it is accumulated, and after the
// rotations Q^T z = R_n .. R_1 y.
// One column (batch column c, global column j) by one warp, V written at Vo.
__device__ void vectors_column(const EigArgs& a, const FactorSrc& f, int c, int j, bool spectra, double* Vo) {
    extern __shared__ __align__(16) double sm[];
    const int lane = threadIdx.x & 31;
    const int nm = a.nu_max, ld = nm + 1;
    const int nu = a.nu_eff[j];
    double* R = sm;                 // reflectors (column k below the diagonal), tau_k on the diagonal
    double* L = R + nm * ld;
    double* Q = L + nm * ld;
    double* inv = Q + nm * ld;
    double* zs = inv + nm;          // [3][nm]: z = Q_H y (spectra only)
    for (int q = lane; q < nu * nu; q += 32) {   // the triangles in use; zero elsewhere
        const int i = q / nu, k = q % nu;
        R[k * ld + i] = k >= i ? f.F[f.rrow(i) + k] : 0.0;
        L[i * ld + k] = k <= i ? f.Lf[f.lrow(i) + k] : 0.0;
        Q[i * ld + k] = (i == k) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int i = lane; i < nu; i += 32) inv[i] = 1.0 / L[i * ld + i];
    // Q_H = H_0 H_1 ... H_{nu-3}, accumulated from the last reflector (rows / columns > k only)
    for (int k = nu - 3; k >= 0; --k) {
        const double tau = R[k * ld + k];
        if (tau == 0.0) continue;
        for (int n = k + 1 + lane; n < nu; n += 32) {
            double t = 0.0;
            for (int i = k + 1; i < nu; ++i) t = fma(R[i * ld + k], Q[i * ld + n], t);
            t *= tau;
            for (int i = k + 1; i < nu; ++i) Q[i * ld + n] = fma(-t, R[i * ld + k], Q[i * ld + n]);
        }
        __syncwarp();
    }
    if (spectra) {   // z = Q_H y (lanes over rows)
        const double* y = a.tri + (size_t)c * eig_tri_doubles(nm) + 2 * nm;
        for (int i = lane; i < nu; i += 32) {
            double z0 = 0.0, z1 = 0.0, z2 = 0.0;
            for (int k = 0; k < nu; ++k) {
                const double q = Q[i * ld + k];
                z0 = fma(q, y[k], z0);
                z1 = fma(q, y[nm + k], z1);
                z2 = fma(q, y[2 * nm + k], z2);
            }
            zs[i] = z0;
            zs[nm + i] = z1;
            zs[2 * nm + i] = z2;
        }
        __syncwarp();
    }
    // Q <- Q R^T for every recorded rotation (columns k, k+1; lanes over rows), the rotation list
    // staged through shared memory 128 at a time with coalesced loads
    const int nrot = f.nrot;
    const double* rc = f.rc;
    const double* rs = f.rs;
    const unsigned char* rk = f.rk;
    __shared__ double sc[kRotStage], ss[kRotStage];
    __shared__ int sk[kRotStage];
    for (int r0 = 0; r0 < nrot; r0 += kRotStage) {
        const int cnt = min(kRotStage, nrot - r0);
        for (int q = lane; q < cnt; q += 32) {
            sc[q] = __ldg(rc + r0 + q);
            ss[q] = __ldg(rs + r0 + q);
            sk[q] = __ldg(rk + r0 + q);
        }
        __syncwarp();
        for (int r = 0; r < cnt; ++r) {
            const double cr = sc[r], sr = ss[r];
            const int k = sk[r];
            for (int q = lane; q < nu; q += 32) {
                const double q0 = Q[q * ld + k], q1 = Q[q * ld + k + 1];
                Q[q * ld + k] = fma(cr, q0, sr * q1);
                Q[q * ld + k + 1] = fma(cr, q1, -sr * q0);
            }
        }
        __syncwarp();
    }
    if (spectra) {   // c, d, g = Q^T z in ascending order of the poles (lanes over poles)
        const int* pm = f.perm;
        for (int k = lane; k < nm; k += 32) {
            double sc = 0.0, sd = 0.0, sg = 0.0;
            if (k < nu) {
                const int p = pm[k];
                for (int n = 0; n < nu; ++n) {
                    const double q = Q[n * ld + p];
                    sc = fma(q, zs[n], sc);
                    sd = fma(q, zs[nm + n], sd);
                    sg = fma(q, zs[2 * nm + n], sg);
                }
            }
            a.c[(size_t)j * nm + k] = sc;
            a.d[(size_t)j * nm + k] = sd;
            a.g[(size_t)j * nm + k] = sg;
        }
    }
    // V = L^-T Q in place (lanes over columns m, rows bottom-up)
    for (int m = lane; m < nu; m += 32)
        for (int i = nu - 1; i >= 0; --i) {
            double s = Q[i * ld + m];
            for (int l = i + 1; l < nu; ++l) s = fma(-L[l * ld + i], Q[l * ld + m], s);
            Q[i * ld + m] = s * inv[i];
        }
    __syncwarp();
    const int* perm = f.perm;
    for (int q = lane; q < nu * nu; q += 32) {
        const int n = q / nu, k = q % nu;
        Vo[(size_t)n * nm + k] = Q[n * ld + perm[k]];
    }
}

__global__ void __launch_bounds__(32) k_eig_vectors(const EigArgs a, bool spectra) {
    const int c = blockIdx.x;
    if (c >= a.ncols) return;
    vectors_column(a, batch_factors(a, c), c, a.col0 + c, spectra, a.V + (size_t)c * a.nu_max * a.nu_max);
}

// the columns of the batch that k_eig_archive listed (the pool could not hold them)
__global__ void __launch_bounds__(32) k_eig_vectors_listed(const EigArgs a) {
    const unsigned long long cnt = a.ar.cnt[2];
    for (unsigned long long q = blockIdx.x; q < cnt; q += gridDim.x) {
        const int c = a.ar.list[q];
        vectors_column(a, batch_factors(a, c), c, a.col0 + c, false, a.V + (size_t)c * a.nu_max * a.nu_max);
        __syncwarp();
    }
}

// every column the archive holds (a.col0 = 0: batch column = global column)
__global__ void __launch_bounds__(32) k_eig_vectors_archived(const EigArgs a) {
    const int j = blockIdx.x;
    if (j >= a.ncols || a.ar.n[j] < 0) return;
    vectors_column(a, archived_factors(a, j), j, j, false, a.V + (size_t)j * a.nu_max * a.nu_max);
}

// ----------------------------------------------------------------------------- k_eig_archive
// One warp per batch column: a run of the pool taken with one atomic (runs land in any order;
// each column reads only its own), the rotations, the two triangles in use and the eigenvalue
// order copied. A column past the pool's end is listed instead, and gets n[j] = -1.
__global__ void __launch_bounds__(128) k_eig_archive(const EigArgs a) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (c >= a.ncols) return;
    const int nm = a.nu_max, j = a.col0 + c, nu = a.nu_eff[j];
    const FactorSrc f = batch_factors(a, c);
    const unsigned long long n = (unsigned long long)f.nrot;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(a.ar.cnt, n);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (off + n > a.ar.cap) {
        if (lane == 0) {
            a.ar.n[j] = -1;
            atomicAdd(a.ar.cnt + 1, 1ull);
            a.ar.list[atomicAdd(a.ar.cnt + 2, 1ull)] = c;
        }
        return;
    }
    for (unsigned long long r = lane; r < n; r += 32) {
        a.ar.rot_c[off + r] = f.rc[r];
        a.ar.rot_s[off + r] = f.rs[r];
        a.ar.rot_k[off + r] = f.rk[r];
    }
    double* F = a.ar.fac + (size_t)j * eig_arch_fac_doubles(nm);
    double* Lp = F + (size_t)nm * (nm + 1) / 2;
    for (int k = 0; k < nu; ++k) {   // rows as archived_factors reads them
        const long long ru = (long long)k * nm - (long long)k * (k - 1) / 2 - k, rl = (long long)k * (k + 1) / 2;
        for (int i = k + lane; i < nu; i += 32) F[ru + i] = f.F[f.rrow(k) + i];
        for (int l = lane; l <= k; l += 32) Lp[rl + l] = f.Lf[f.lrow(k) + l];
    }
    for (int k = lane; k < nu; k += 32) a.ar.perm[(size_t)j * nm + k] = f.perm[k];
    if (lane == 0) {
        a.ar.n[j] = (int)n;
        a.ar.off[j] = off;
    }
}

// ----------------------------------------------------------------------------- k_eig_weights
// t = V w for the density weights of Eq. 2, w = 2 f(e_k - mu) c_k and w e_k, without V:
// V w = L^-T Q_H R_1^T .. R_n^T w (w put back in the order of the eigenvalue iteration). In turn:
//   the recorded rotations in reverse, each turning (w_k, w_k+1) into (c w_k - s w_k+1,
//   s w_k + c w_k+1);
//   the reflectors H_{nu-3} .. H_0, H_k x = x - tau_k v_k (v_k^T x);
//   the back substitution L^T t = x (t_i = x_i / L_ii, then x_l -= L_il t_i for l < i).
// One thread per (column, vector): a CTA takes 32 columns, warp 0 the vector w, warp 1 w e. No
// reductions across lanes, so every FP64 instruction carries 32 columns.
// Out: T[batch col][2 nu_max] = (t, t_E), zero past nu. kArch: every column from the archive
// (a.col0 = 0), and t = V w from the stored V (a.V) for a column whose V was formed instead.
constexpr int kWtThreads = 64;
template <bool kArch>
__global__ void __launch_bounds__(kWtThreads) k_eig_weights(const EigArgs a, double mu_in, const double* mu_dev,
                                                             double kT, double* T) {
    const double mu = mu_dev ? *mu_dev : mu_in;
    extern __shared__ double csm[];
    const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;
    const int c0 = blockIdx.x * 32, c = c0 + lane;
    const int nm = a.nu_max;
    const Strided<kWtThreads> X{csm + threadIdx.x};
    if (c < a.ncols && kArch && a.ar.n[a.col0 + c] < 0) {
        // w in pole order against V's columns; the thread's own slots of T hold t meanwhile
        const int j = a.col0 + c;
        const int nu = a.nu_eff[j];
        const double* Vj = a.V + (size_t)j * nm * nm;
        double* Tt = T + (size_t)c * 2 * nm + (size_t)v * nm;
        for (int k = 0; k < nm; ++k) X[k] = 0.0;
        for (int k = 0; k < nu; ++k) {
            const double e = a.eps[(size_t)j * nm + k];
            const double f2 = 2.0 * fermi((e - mu) / kT) * a.c[(size_t)j * nm + k];
            X[k] = v ? f2 * e : f2;
        }
        for (int n = 0; n < nu; ++n) {
            double t = 0.0;
            for (int k = 0; k < nu; ++k) t = fma(Vj[(size_t)n * nm + k], X[k], t);
            Tt[n] = t;
        }
        for (int n = 0; n < nu; ++n) X[n] = Tt[n];
    } else if (c < a.ncols) {
        const int j = a.col0 + c;
        const int nu = a.nu_eff[j];
        const FactorSrc fs = kArch ? archived_factors(a, j) : batch_factors(a, c);
        for (int k = 0; k < nm; ++k) X[k] = 0.0;
        const int* perm = fs.perm;
        for (int k = 0; k < nu; ++k) {
            const double e = a.eps[(size_t)j * nm + k];
            const double f2 = 2.0 * fermi((e - mu) / kT) * a.c[(size_t)j * nm + k];
            X[perm[k]] = v ? f2 * e : f2;
        }
        // in reverse; the loads of four rotations issued before the four are applied
        int r = fs.nrot - 1;
        for (; r >= 3; r -= 4) {
            double cq[4], sq[4];
            int kq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cq[q] = __ldg(fs.rc + r - q);
                sq[q] = __ldg(fs.rs + r - q);
                kq[q] = __ldg(fs.rk + r - q);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = kq[q];
                const double p = X[k], w = X[k + 1];
                X[k] = fma(cq[q], p, -sq[q] * w);
                X[k + 1] = fma(cq[q], w, sq[q] * p);
            }
        }
        for (; r >= 0; --r) {
            const double cr = __ldg(fs.rc + r), sr = __ldg(fs.rs + r);
            const int k = __ldg(fs.rk + r);
            const double p = X[k], w = X[k + 1];
            X[k] = fma(cr, p, -sr * w);
            X[k + 1] = fma(cr, w, sr * p);
        }
        for (int k = nu - 3; k >= 0; --k) {
            const double* vk = fs.F + fs.rrow(k);
            const double tau = vk[k];
            if (tau == 0.0) continue;
            double s0 = 0.0, s1 = 0.0;           // two partial sums: half the dependent chain
            int i = k + 1;
            for (; i + 1 < nu; i += 2) {
                s0 = fma(vk[i], X[i], s0);
                s1 = fma(vk[i + 1], X[i + 1], s1);
            }
            if (i < nu) s0 = fma(vk[i], X[i], s0);
            const double sc = tau * (s0 + s1);
            for (int m = k + 1; m < nu; ++m) X[m] = fma(-sc, vk[m], X[m]);
        }
        for (int i = nu - 1; i >= 0; --i) {
            const double* row = fs.Lf + fs.lrow(i);
            const double ti = X[i] / row[i];
            X[i] = ti;
            for (int l = 0; l < i; ++l) X[l] = fma(-row[l], ti, X[l]);
        }
    }
    __syncthreads();
    // coalesced write-out: element k of vector v of column c0 + t sits at csm[k * 64 + v * 32 + t]
    const int ncl = min(32, a.ncols - c0);
    for (int q = threadIdx.x; q < ncl * 2 * nm; q += kWtThreads) {
        const int t = q / (2 * nm), r = q % (2 * nm);
        const int vv = r / nm, k = r % nm;
        T[(size_t)(c0 + t) * 2 * nm + r] = csm[(size_t)k * kWtThreads + vv * 32 + t];
    }
}

// The largest dynamic shared memory any eigensolver kernel asks for at capacity nm (checked
// against the device before the columns are planned).
size_t eig_smem_max(int nm);

size_t eig_smem_reduce(int nm) {
    return sizeof(double) * 2 * ((2 * (size_t)nm + 3) * (nm + 1) + 2 * (size_t)nm + 3);
}
size_t eig_smem_vectors(int nm) { return sizeof(double) * (3 * (size_t)nm * (nm + 1) + 4 * (size_t)nm); }
size_t eig_smem_threads(int nm, int arrays) { return sizeof(double) * arrays * (size_t)nm * kChaseThreads; }
size_t eig_smem_max(int nm) {
    const size_t spec = sizeof(double) * (size_t)nm * kSpecThreads, wt = sizeof(double) * (size_t)nm * kWtThreads;
    return std::max({eig_smem_reduce(nm), eig_smem_vectors(nm), eig_smem_threads(nm, 2), spec, wt});
}
int eig_thread_grid(int ncols) { return (ncols + kChaseThreads - 1) / kChaseThreads; }

void projected_eig(const EigArgs& a, cudaStream_t st, bool form_v) {
    const size_t s1 = eig_smem_reduce(a.nu_max);
    smem_at_least(k_eig_reduce, s1);
    k_eig_reduce<<<(a.ncols + 1) / 2, 64, s1, st>>>(a);
    const size_t s2 = eig_smem_threads(a.nu_max, 2);
    smem_at_least(k_eig_chase, s2);
    carveout_for(k_eig_chase, s2, eig_thread_grid(a.ncols));
    k_eig_chase<<<eig_thread_grid(a.ncols), kChaseThreads, s2, st>>>(a);
    const size_t sv = eig_smem_vectors(a.nu_max);
    smem_at_least(k_eig_vectors, sv);
    if (form_v) {   // V and the spectra in one kernel
        k_eig_vectors<<<a.ncols, 32, sv, st>>>(a, true);
        return;
    }
    const size_t s3 = sizeof(double) * (size_t)a.nu_max * kSpecThreads;
    smem_at_least(k_eig_spectra, s3);
    carveout_for(k_eig_spectra, s3, (a.ncols + 31) / 32, kStreamCtas);
    k_eig_spectra<<<(a.ncols + 31) / 32, kSpecThreads, s3, st>>>(a);
}

void eig_vectors(const EigArgs& a, cudaStream_t st) {   // the spectra in use are kept
    const size_t s = eig_smem_vectors(a.nu_max);
    smem_at_least(k_eig_vectors, s);
    k_eig_vectors<<<a.ncols, 32, s, st>>>(a, false);
}

void eig_density_weights(const EigArgs& a, double mu, const double* mu_dev, double kT, double* T, cudaStream_t st) {
    const size_t s = sizeof(double) * (size_t)a.nu_max * kWtThreads;
    smem_at_least(k_eig_weights<false>, s);
    carveout_for(k_eig_weights<false>, s, (a.ncols + 31) / 32, kStreamCtas);
    k_eig_weights<false><<<(a.ncols + 31) / 32, kWtThreads, s, st>>>(a, mu, mu_dev, kT, T);
}

void eig_archive(const EigArgs& a, cudaStream_t st) {
    cudaMemsetAsync(a.ar.cnt + 2, 0, sizeof(unsigned long long), st);
    k_eig_archive<<<(a.ncols + 3) / 4, 128, 0, st>>>(a);
    const size_t sv = eig_smem_vectors(a.nu_max);
    smem_at_least(k_eig_vectors_listed, sv);
    k_eig_vectors_listed<<<std::max(1, std::min(a.ncols, 2048)), 32, sv, st>>>(a);
}

void eig_vectors_archived(const EigArgs& a, cudaStream_t st) {
    const size_t sv = eig_smem_vectors(a.nu_max);
    smem_at_least(k_eig_vectors_archived, sv);
    k_eig_vectors_archived<<<a.ncols, 32, sv, st>>>(a);
}

void eig_density_weights_archived(const EigArgs& a, double mu, const double* mu_dev, double kT, double* T,
                                  cudaStream_t st) {
    const size_t s = sizeof(double) * (size_t)a.nu_max * kWtThreads;
    smem_at_least(k_eig_weights<true>, s);
    carveout_for(k_eig_weights<true>, s, (a.ncols + 31) / 32, kStreamCtas);
    k_eig_weights<true><<<(a.ncols + 31) / 32, kWtThreads, s, st>>>(a, mu, mu_dev, kT, T);
}

}  // namespace elses
