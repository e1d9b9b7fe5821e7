// a5 + a6: projected generalized eigenproblem H' v = e S' v per column, and its spectra.
//
// Eq. 1 is solved instead of the generalized eigenvalue equation H y = e S y of the whole
// system; on the nu-dimensional Krylov space of a column that equation is small and is solved
// exactly:  S' = L L^T (Cholesky),  A = L^-1 H' L^-T,  A = Q diag(e) Q^T,  V = L^-T Q.
// The Green's-function column then has poles e_k and residues Z_ik c_k with Z = U V and
// c = V^T U^T e_j; kept per column are (e, c, d = V^T (SU)_j, g = V^T (HU)_j) and V.
//
// GB300 form: one thread per column (the problem is small, sequential and FP64; spreading it
// over a warp would repeat its scalar recurrences on every lane of the FP64 pipe). Each
// thread's matrices live in global memory in [element][column] order, so the 32 threads of a
// warp touch consecutive addresses. Symmetric eigensolver: Householder reduction to
// tridiagonal form, then implicit-shift QR sweeps (Wilkinson shift, Givens bulge chase) with
// the rotations accumulated into Q; eigenvalues sorted ascending.
#include "internal.h"

namespace elses {

size_t eig_work_doubles(int nu_max) { return 3 * (size_t)nu_max * nu_max + 6 * (size_t)nu_max; }

__global__ void k_proj_eig(const EigArgs a) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.ncols) return;
    const int j = a.col0 + c;
    const int nu = a.nu_eff[j];
    const int nm = a.nu_max;
    const size_t st = a.ncols_pad;
    double* W = a.work + c;
    const size_t oA = 0, oQ = (size_t)nm * nm, oL = 2 * (size_t)nm * nm, oD = 3 * (size_t)nm * nm;
    const size_t oE = oD + nm, oT = oE + nm, oP = oT + nm, oI = oP + nm, oX = oI + nm;
#define AM(i, k) W[(oA + (size_t)(i) * nm + (k)) * st]
#define QM(i, k) W[(oQ + (size_t)(i) * nm + (k)) * st]
#define LM(i, k) W[(oL + (size_t)(i) * nm + (k)) * st]
#define DV(i) W[(oD + (i)) * st]
#define EV(i) W[(oE + (i)) * st]
#define TV(i) W[(oT + (i)) * st]
#define PV(i) W[(oP + (i)) * st]
#define IV(i) W[(oI + (i)) * st]
#define XV(i) W[(oX + (i)) * st]
    const int PK = nm * (nm + 1) / 2;
    const double* Hp = a.Hp + (size_t)c * PK;
    const double* Sp = a.Sp + (size_t)c * PK;
    // packed upper storage: element (i, k), i <= k, at i + k (k + 1) / 2
#define PACK(P, i, k) ((i) <= (k) ? (P)[(i) + (k) * ((k) + 1) / 2] : (P)[(k) + (i) * ((i) + 1) / 2])

    // 1. Cholesky of S'
    for (int i = 0; i < nu; ++i) {
        for (int k = 0; k <= i; ++k) {
            double s = PACK(Sp, i, k);
            for (int m = 0; m < k; ++m) s -= LM(i, m) * LM(k, m);
            if (i == k) {
                if (!(s > 0.0)) {
                    flag(a.status, DEV_NOT_SPD);
                    return;
                }
                const double l = sqrt(s);
                LM(i, i) = l;
                IV(i) = 1.0 / l;
            } else {
                LM(i, k) = s * IV(k);
            }
        }
    }
    // 2. X = L^-1 H' (kept in Q), 3. Y = L^-1 X^T (kept in A), A = (Y + Y^T) / 2
    for (int n = 0; n < nu; ++n)
        for (int i = 0; i < nu; ++i) {
            double s = PACK(Hp, i, n);
            for (int m = 0; m < i; ++m) s -= LM(i, m) * QM(m, n);
            QM(i, n) = s * IV(i);
        }
    for (int n = 0; n < nu; ++n)
        for (int i = 0; i < nu; ++i) {
            double s = QM(n, i);
            for (int m = 0; m < i; ++m) s -= LM(i, m) * AM(m, n);
            AM(i, n) = s * IV(i);
        }
    for (int i = 0; i < nu; ++i)
        for (int k = 0; k < i; ++k) {
            const double v = 0.5 * (AM(i, k) + AM(k, i));
            AM(i, k) = v;
            AM(k, i) = v;
        }
    // 4. Householder tridiagonalisation, Q accumulated
    for (int i = 0; i < nu; ++i)
        for (int k = 0; k < nu; ++k) QM(i, k) = (i == k) ? 1.0 : 0.0;
    for (int k = 0; k + 2 < nu; ++k) {
        double sigma = 0.0;
        for (int i = k + 1; i < nu; ++i) sigma += AM(i, k) * AM(i, k);
        const double x0 = AM(k + 1, k);
        if (sigma == 0.0) continue;
        const double alpha = -copysign(sqrt(sigma), x0);
        const double tau = 1.0 / (alpha * (alpha - x0));   // 2 / ||v||^2
        TV(k + 1) = x0 - alpha;
        for (int i = k + 2; i < nu; ++i) TV(i) = AM(i, k);
        double K = 0.0;
        for (int i = k + 1; i < nu; ++i) {
            double s = 0.0;
            for (int m = k + 1; m < nu; ++m) s += AM(i, m) * TV(m);
            PV(i) = tau * s;
            K += TV(i) * PV(i);
        }
        K *= 0.5 * tau;
        for (int i = k + 1; i < nu; ++i) PV(i) -= K * TV(i);
        for (int i = k + 1; i < nu; ++i)
            for (int m = k + 1; m < nu; ++m) AM(i, m) -= TV(i) * PV(m) + PV(i) * TV(m);
        AM(k + 1, k) = alpha;
        AM(k, k + 1) = alpha;
        for (int i = k + 2; i < nu; ++i) { AM(i, k) = 0.0; AM(k, i) = 0.0; }
        for (int r = 0; r < nu; ++r) {
            double t = 0.0;
            for (int m = k + 1; m < nu; ++m) t += QM(r, m) * TV(m);
            t *= tau;
            for (int m = k + 1; m < nu; ++m) QM(r, m) -= t * TV(m);
        }
    }
    for (int i = 0; i < nu; ++i) DV(i) = AM(i, i);
    for (int i = 0; i + 1 < nu; ++i) EV(i) = AM(i + 1, i);
    // 5. implicit-shift QR on the tridiagonal (D, E)
    const double eps = 2.220446049250313e-16;
    int hi = nu - 1, sweeps = 0;
    while (hi > 0) {
        if (fabs(EV(hi - 1)) <= eps * (fabs(DV(hi - 1)) + fabs(DV(hi)))) {
            EV(hi - 1) = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && fabs(EV(lo - 1)) > eps * (fabs(DV(lo - 1)) + fabs(DV(lo)))) --lo;
        if (lo > 0) EV(lo - 1) = 0.0;
        if (++sweeps > 30 * nu) {
            flag(a.status, DEV_TIMEOUT);
            break;
        }
        const double delta = 0.5 * (DV(hi - 1) - DV(hi));
        const double b2 = EV(hi - 1) * EV(hi - 1);
        const double den = delta + copysign(sqrt(delta * delta + b2), delta);
        const double mu = DV(hi) - (den != 0.0 ? b2 / den : 0.0);
        double x = DV(lo) - mu, z = EV(lo);
        for (int k = lo; k < hi; ++k) {
            const double r = hypot(x, z);
            double cr = 1.0, sr = 0.0;
            if (r != 0.0) { cr = x / r; sr = z / r; }
            if (k > lo) EV(k - 1) = r;
            const double ak = DV(k), ak1 = DV(k + 1), b = EV(k);
            const double cc = cr * cr, ss = sr * sr, cs = cr * sr;
            DV(k) = cc * ak + 2.0 * cs * b + ss * ak1;
            DV(k + 1) = ss * ak - 2.0 * cs * b + cc * ak1;
            EV(k) = cs * (ak1 - ak) + (cc - ss) * b;
            if (k + 1 < hi) {
                const double bn = EV(k + 1);
                z = sr * bn;
                EV(k + 1) = cr * bn;
                x = EV(k);
            }
            for (int q = 0; q < nu; ++q) {
                const double qk = QM(q, k), qk1 = QM(q, k + 1);
                QM(q, k) = cr * qk + sr * qk1;
                QM(q, k + 1) = -sr * qk + cr * qk1;
            }
        }
    }
    // 6. ascending order (selection, columns of Q follow)
    for (int k = 0; k + 1 < nu; ++k) {
        int m = k;
        for (int q = k + 1; q < nu; ++q)
            if (DV(q) < DV(m)) m = q;
        if (m != k) {
            const double t = DV(k); DV(k) = DV(m); DV(m) = t;
            for (int q = 0; q < nu; ++q) { const double u = QM(q, k); QM(q, k) = QM(q, m); QM(q, m) = u; }
        }
    }
    // 7. V = L^-T Q (back substitution, kept in A), spectra
    for (int k = 0; k < nu; ++k)
        for (int i = nu - 1; i >= 0; --i) {
            double s = QM(i, k);
            for (int m = i + 1; m < nu; ++m) s -= LM(m, i) * AM(m, k);
            AM(i, k) = s * IV(i);
        }
    const double* ur = a.urow + (size_t)c * nm;
    const double* sr = a.surow + (size_t)c * nm;
    const double* hr = a.hurow + (size_t)c * nm;
    double* Vo = a.V + (size_t)c * nm * nm;
    for (int k = 0; k < nm; ++k) {
        double cc = 0.0, dd = 0.0, gg = 0.0, e = 0.0;
        if (k < nu) {
            for (int n = 0; n < nu; ++n) {
                const double v = AM(n, k);
                cc += v * ur[n];
                dd += v * sr[n];
                gg += v * hr[n];
                Vo[(size_t)n * nm + k] = v;
            }
            e = DV(k);
        }
        a.eps[(size_t)j * nm + k] = e;
        a.c[(size_t)j * nm + k] = cc;
        a.d[(size_t)j * nm + k] = dd;
        a.g[(size_t)j * nm + k] = gg;
    }
#undef AM
#undef QM
#undef LM
#undef DV
#undef EV
#undef TV
#undef PV
#undef IV
#undef XV
#undef PACK
}

void projected_eig(const EigArgs& a, cudaStream_t st) {
    const int T = 64;
    k_proj_eig<<<(a.ncols + T - 1) / T, T, 0, st>>>(a);
}

}  // namespace elses
