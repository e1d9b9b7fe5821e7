// Internal declarations shared by the translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace elses {

struct CellGrid {
    int nc[3];
    double len[3];
    double L[3];
    int ncell;
};

// ---------------------------------------------------------------- a1 (neighbors.cu)
void scan_exclusive(const int* in, int* out, int n, cudaStream_t st);
void build_cells(const double* pos, int n, const CellGrid& g, int* cell_of, int* cell_count,
                 int* cell_start, int* cursor, int* cell_atoms, cudaStream_t st);
void count_lists(const double* pos, int n, const CellGrid& g, const int* cell_of,
                 const int* cell_start, const int* cell_atoms, double r, int* counts,
                 int* max_count, cudaStream_t st);
void fill_lists(const double* pos, int n, const CellGrid& g, const int* cell_of,
                const int* cell_start, const int* cell_atoms, double r, const int* ptr, int* idx,
                int cap, int* status, cudaStream_t st);
// count += the pattern pairs (I, J), I in row J, with I outside the cluster of J
void pattern_outside_clusters(int n, const int* row_ptr, const int* col_idx, const int* cl_ptr,
                              const int* cl_idx, int* count, cudaStream_t st);

// Sets the thread-local message returned by elses_last_error and returns `code`.
int report_error(int code, const char* fmt, ...);

void check_finite(const double* x, int count, int* status, cudaStream_t st);
int probe_fp64(double* gflops, cudaStream_t st);   // returns a cudaError_t value

// ---------------------------------------------------------------- a2, a10 (sk_build.cu)
void sk_build(const double* pos, int n, const double L[3], const SKDev& sk, const int* row_ptr,
              const int* col_idx, int nnzb, int* row_of, int* tmap, double* H, double* S,
              double* skr, cudaStream_t st);
void forces(const double* pos, int n, const double L[3], const SKDev& sk, const int* row_ptr,
            const int* col_idx, const int* row_of, const int* tmap, int nnzb, const double* rho,
            const double* rhoE, double* g_block, double* F, cudaStream_t st);
void icohp(const double* pos, const double L[3], const SKDev& sk, const int* col_idx, const int* row_of,
           int nnzb, const double* H, const double* rho, double* B, double* Bsig, double* Bpi, cudaStream_t st);
void cohp_spectrum(const double* pos, const double L[3], const SKDev& sk, const int* col_idx, const int* row_of,
                   int nnzb, const double* H, const double* G, int n_zc, int iz0, int n_z, double* C,
                   double* Csig, double* Cpi, cudaStream_t st);

// ---------------------------------------------------------------- a3, a4 (krylov.cu)
struct KrylovArgs {
    int n_atoms;
    const int* row_ptr;
    const int* col_idx;
    const double* H;
    const double* S;
    const double* skr;      // two-centre records [nnzb][12] (u, H and S integrals) or nullptr
    const int* cl_ptr;      // nullptr: every cluster is the whole system
    const int* cl_idx;
    int atom_begin, atom_end;
    const int* order;       // atoms of this launch in processing order (n_items of them)
    int n_items;
    int* queue;             // optional: work counter of the persistent queue (batched form)
    int nu_max;             // allocation stride of per-column Krylov arrays
    int nu_default;
    int n_classes;
    int class_max_atoms[4];
    int class_nu[4];
    double breakdown_tol;
    int reorth;             // 1: second-pass coefficients from S' (elses_params.reorth)
    int onsite_diag;        // 1: on-site S blocks are I and on-site H blocks diagonal
    int na_max;             // cluster capacity: a multiple of 32 (of 16 with half)
    int half;               // 1: two columns per warp, one per half-warp (k_krylov_half)
    int deg_max;            // maximum pattern row length
    double* scratch;        // per resident CTA: 4 warps x (U, SU) x nu_max x na_max x 4
    double* Hp;             // [col][nu_max*(nu_max+1)/2] packed upper, batch-local col
    double* Sp;
    double* urow;           // [col][nu_max]: row j of U, SU, HU
    double* surow;
    double* hurow;
    int* nu_eff;            // [M] global
    double* UP;             // pattern rows of U: [(e*4 + alpha)*4 + r][nu_max], e - up_block0
    int up_block0;
    int* status;
    unsigned long long* flops;   // algorithmic FP64 flops of the columns, accumulated
    // optional per-column store of the bases for the exact gradient (nullptr: not kept):
    // column j at bstore + j * bstride holds U, SU, HU (bvec doubles apart), then the
    // Gram-Schmidt coefficients [nu_max][nu_max] and H' packed upper
    double* bstore;
    size_t bstride, bvec;
};

// Exact-gradient pass (adjoint.cu) over the columns of a batch; the KrylovArgs of the same batch
// drive the recomputed forward recursion.
struct AdjointArgs {
    const double* V;        // [col - v_col0][nu_max][nu_max] eigenvectors (rows: Krylov index)
    int v_col0;
    const double* eps;      // [M][nu_max] poles ascending, and the spectra c, d
    const double* c;
    const double* d;
    double mu, kT;
    const double* mu_dev;   // when set, mu is read here (device) instead
    // dOmega/dH and dOmega/dS accumulated as exact 128-bit fixed-point sums ([2][nnzb * 16]
    // pairs (low, high word) of unsigned 64-bit words, value * 2^80 in two's complement): integer
    // addition is associative, so the sums do not depend on the order of the atomics
    unsigned long long* acc;
    int nnzb;
    unsigned long long* flops;   // algorithmic FP64 flops of the gradient kernels, accumulated
    int* status;
    double* scratch;        // per resident CTA: 4 warps x adjoint_warp_doubles(nu_max, na_max)
    int atom_lo, atom_hi;   // only atoms in [atom_lo, atom_hi) are accumulated
    const double* bstore;   // bases kept by the energy pass (KrylovArgs layout), or nullptr:
    size_t bstride, bvec;   // then the forward recursion is recomputed
};
size_t krylov_smem_bytes(int na_max, int deg_max);
int krylov_blocks_per_sm(int na_max, int deg_max);       // resident CTAs at the 3-CTA register budget
int krylov_blocks_per_sm_max(int na_max, int deg_max);   // with the 4-CTA form where shared memory allows
int krylov_half_blocks_per_sm(int na_max, int deg_max);
size_t block_krylov_scratch_doubles(int nu_max, int na_max);
int block_krylov_blocks_per_sm(int na_max, int deg_max);
void block_krylov_columns(const KrylovArgs& a, int grid, cudaStream_t st);
__host__ __device__ size_t adjoint_warp_doubles(int nu_max, int na_max);
int adjoint_blocks_per_sm(int na_max, int deg_max);
void adjoint_columns(const KrylovArgs& a, const AdjointArgs& g, int grid, cudaStream_t st);
// gH = value of acc[0], gS = s_scale * value of acc[1] as doubles ([nnzb * 16] each)
void adjoint_finish(const unsigned long long* acc, size_t n, double s_scale, double* gH, double* gS,
                    cudaStream_t st);
void krylov_columns(const KrylovArgs& a, int grid, int ctas_per_sm, cudaStream_t st);

// ---------------------------------------------------------------- a5, a6 (proj_eig.cu)
// The eigen-factors of every column kept across batches (several batches, stored workflow), so
// that V need not be formed per batch: per global column j the reflectors with tau_k (packed
// upper triangle, row k from entry k) then L (packed lower triangle), nu_max (nu_max + 1)
// doubles; the ascending order of the eigenvalues; and the recorded rotations in a pool shared by
// all columns, each column's run at off[j]. A column whose rotations do not fit in the pool gets
// n[j] = -1 and its V formed instead.
struct FactorArchive {
    double* fac;                 // [M][nu_max (nu_max + 1)]
    int* perm;                   // [M][nu_max]
    int* n;                      // [M]: rotations kept, or -1 (V formed)
    unsigned long long* off;     // [M]: first rotation in the pool
    double* rot_c;               // [cap]
    double* rot_s;
    unsigned char* rot_k;
    unsigned long long cap;      // pool capacity (rotations)
    unsigned long long* cnt;     // device counters: [0] pool use, [1] columns with V formed, [2] this batch's list length
    int* list;                   // [batch cols]: this batch's columns whose V is formed
};
__host__ __device__ size_t eig_arch_fac_doubles(int nm);

struct EigArgs {
    int ncols;              // batch columns
    int col0;               // global index of the first batch column
    int nu_max;
    const double* Hp;
    const double* Sp;
    const double* urow;
    const double* surow;
    const double* hurow;
    const int* nu_eff;      // [M] global
    double* tri;            // [col][5 nu_max]: tridiagonal D, E and the three vectors y = Q_H^T z
    double* fac;            // [col][2 nu_max^2]: Householder reflectors (row k) + tau, Cholesky factor
    double* rot_c;          // [col][rot_cap]: recorded Givens rotations
    double* rot_s;
    unsigned char* rot_k;
    int* rot_n;             // [col]
    int* perm;              // [col][nu_max]: ascending order of the eigenvalues
    double* eps;            // [M][nu_max] global
    double* c;
    double* d;
    double* g;
    double* V;              // [batch col][nu_max*nu_max] (row n = Krylov index, col k = eigen index)
    int* status;
    int max_sweeps;         // QR sweeps allowed per column (0: 30 nu; DEV_TIMEOUT beyond)
    FactorArchive ar;       // the kept factors (several batches), else all null
};
__host__ __device__ size_t eig_tri_doubles(int nm);
__host__ __device__ size_t eig_fac_doubles(int nm);
__host__ __device__ size_t eig_rot_cap(int nm);
// reduce, chase, spectra (eps, c, d, g); V too when form_v
void projected_eig(const EigArgs& a, cudaStream_t st, bool form_v);
size_t eig_smem_max(int nm);   // largest dynamic shared memory of the eigensolver kernels
// V of the columns whose factors (fac, rotations, perm) are those of the last projected_eig
void eig_vectors(const EigArgs& a, cudaStream_t st);
// T[batch col][2 nu_max]: t = V w and t_E = V w_E for the density weights at mu, from the factors
void eig_density_weights(const EigArgs& a, double mu, const double* mu_dev, double kT, double* T, cudaStream_t st);
// the batch's factors into the archive (a.ar), then V (at a.V) of its columns the pool cannot hold
void eig_archive(const EigArgs& a, cudaStream_t st);
// every column from the archive (a.col0 = 0, a.ncols = M, a.V the stored V): V of the columns
// kept there; T[M][2 nu_max] for the density weights at mu (from V where it was formed instead)
void eig_vectors_archived(const EigArgs& a, cudaStream_t st);
void eig_density_weights_archived(const EigArgs& a, double mu, const double* mu_dev, double kT, double* T,
                                  cudaStream_t st);

// ---------------------------------------------------------------- a7, a9 (reduce.cu)
struct BisectState {
    double lo, hi, mu;
    double n_lo, n_hi, n_mid;
    double n_at, e_band, omega;
    double mu0;             // where the kept exponentials were taken
    double scale;           // exp((mu0 - x)/kT) at the next midpoint x, once they are kept
    int iter, done, status, have_pre;
};
struct ReduceArgs {
    int M;
    int nu_max;
    const double* eps;
    const double* c;
    const double* d;
    const double* g;
    const int* nu_eff;
    double kT;
    double inv_kT;          // 1 / kT (host-computed: not one division per thread)
    double n_electrons;
    double tol;
    int max_iter;
    BisectState* state;
    double* partials;       // [grid][4]
    unsigned* ticket;
    // optional, kept by the bisection once its bracket is narrow: per block of k_count, the poles
    // within 60 kT of mu0 as (exp((e - mu0)/kT), d c) in its own range of act ([M][nu_max] in
    // all), their number, and the sum of 2 d c of the poles below that window
    double2* act;
    int* act_n;             // [grid]
    double* act_below;      // [grid]
};
int reduce_grid();
void bisect_init(const ReduceArgs& a, cudaStream_t st);      // bracket + N(lo), N(hi)
void bisect_step(const ReduceArgs& a, cudaStream_t st);      // one bisection step (no-op when done)
void scalars_at(const ReduceArgs& a, double mu, cudaStream_t st);  // N, E_band, Omega at mu
void scalars_at_state(const ReduceArgs& a, cudaStream_t st);      // the same at the state's mu
// DOS at n_z energies; scratch holds dos_scratch_doubles(n_z), the result in its last n_z
size_t dos_scratch_doubles(int n_z);
void dos_at(const ReduceArgs& a, const double* z_dev, int n_z, double* scratch, cudaStream_t st);

// ---------------------------------------------------------------- a8, G(z) (density.cu)
struct DensityArgs {
    int atom_begin, atom_end;
    const int* row_ptr;
    const int* tmap;
    int nu_max;
    const double* eps;      // [M][nu_max] global
    const double* c;
    const int* nu_eff;
    const double* V;        // batch-local columns
    int v_col0;             // global column of V's (or T's and fac's) first column
    const double* T;        // t = V w, t_E [batch col][2 nu_max] (k_eig_weights); used instead of V when set
    const double* UP;
    int up_block0;
    double mu, kT;
    const double* mu_dev;   // when set, mu is read here (device) instead
    double* rho;
    double* rhoE;
    int n_z;
    const double* z;        // device [n_z][2]
    double* G;              // [(e*16 + a*4 + b)*n_z + iz][2]
};
void density_columns(const DensityArgs& a, cudaStream_t st);
void green_columns_eval(const DensityArgs& a, cudaStream_t st);

}  // namespace elses
