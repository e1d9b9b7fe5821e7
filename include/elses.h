/*
 * elses.h -- C ABI of the GB300 per-column Krylov Green's-function library.
 *
 * The library computes, for sparse real-symmetric LCAO matrices H and S (S positive definite),
 * the Green's function G = (zS - H)^-1 column by column (Eq. 1 with b = e_j, the column index
 * j being the parallel unit), the one-body density matrix of Eq. 2 from the Fermi-Dirac energy
 * integral of Im G, the chemical potential by bisection (the workflow of Eq. 3), the band energy
 * Tr(rho H) (= sum of ICOHP, Eq. 6) and the atomic forces, for a two-centre s/p tight-binding
 * model of carbon.
 *
 * Conventions
 *   Units      eV, Angstrom. All floating point is IEEE double (FP64).
 *   Basis      N atoms, M = 4N orbitals; basis index j = 4*J + alpha, alpha = (s, px, py, pz).
 *   Positions  double[N][3], row-major; orthorhombic periodic box; minimum-image convention
 *              (the box must exceed 2*r_cut, and 2*r_cluster when r_cluster > 0).
 *   Pattern    block-sparse rows (BSR) over atoms: row_ptr int32[N+1], col_idx int32[nnzb]
 *              (ascending within a row, the diagonal block included); block e = (I, J) holds
 *              val[e][a][b] = X_(I,a),(J,b) as double[nnzb][4][4]. The pattern is every pair with
 *              |R_J - R_I| <= r_cut (inclusive), so it is symmetric.
 *   Memory     Array arguments named *_dev are caller-owned DEVICE pointers (e.g. from PyTorch),
 *              valid for the duration of the call; *_host are host pointers. Opaque handles and
 *              the device memory behind them are owned by the library and released by
 *              elses_system_destroy; the elses_get_* accessors copy out of that memory.
 *   Streams    Every call takes a cudaStream_t (passed as void*; NULL = legacy default stream)
 *              and enqueues its work on it. Calls that return host scalars synchronise that
 *              stream before returning.
 *   Status     0 = success; > 0 = warning (results valid); < 0 = error (outputs undefined).
 *              elses_last_error() returns a message for the last failing call of this thread.
 *   Threads    One system handle must not be used from two threads at once.
 */
#ifndef ELSES_H
#define ELSES_H

#ifdef __cplusplus
extern "C" {
#endif

#define ELSES_OK                  0
#define ELSES_WARN_BREAKDOWN      1   /* some column stopped early (invariant subspace) */
#define ELSES_ERR_ARG            -1   /* bad argument (NULL, size, box too small, ...)   */
#define ELSES_ERR_NOT_SPD        -2   /* S is not positive definite: a Krylov vector w
                                         with w^T S w < -(breakdown_tol ||H u_n||)^2, or a
                                         projected overlap S' that fails its Cholesky     */
#define ELSES_ERR_NONFINITE      -3   /* NaN or Inf in an input or a result              */
#define ELSES_ERR_NO_BRACKET     -4   /* electron count not bracketed by the spectrum    */
#define ELSES_ERR_TIMEOUT        -5   /* a bounded device-side iteration ran out         */
#define ELSES_ERR_CUDA           -6   /* CUDA runtime error                              */
#define ELSES_ERR_OOM            -7   /* device allocation failed                        */
#define ELSES_ERR_NOT_IMPLEMENTED -8
#define ELSES_ERR_STATE          -9   /* call out of order (e.g. density before columns) */
#define ELSES_ERR_CAPACITY      -10   /* a neighbour or cluster list exceeded its bound,
                                         or a kernel would need more shared memory than
                                         the device has (cluster size, Krylov dimension) */

/* Two-centre s/p Slater-Koster model (reading of the paper's TB-form Hamiltonian):
 * integral x in (ss-sigma, sp-sigma, pp-sigma, pp-pi),
 *   V_x(r) = V0[x] exp(-qH[x] (r - r0)) t(r),   S_x(r) = S0[x] exp(-qS[x] (r - r0)) t(r),
 *   t = 1 (r <= r_on), 0 (r >= r_cut), 1 - 10s^3 + 15s^4 - 6s^5 between, s = (r-r_on)/(r_cut-r_on).
 * On-site blocks: H = diag(Es, Ep, Ep, Ep), S = I. */
typedef struct elses_sk {
    double Es, Ep;
    double V0[4], qH[4];
    double S0[4], qS[4];
    double r0, r_on, r_cut;
} elses_sk;

/* Method settings. nu is the Krylov dimension per column; when n_classes > 0 the dimension of
 * a column is class_nu[c] for the first class c with cluster atoms <= class_max_atoms[c]. */
typedef struct elses_params {
    double r_cluster;       /* cluster radius around atom J; <= 0: the whole system          */
    double kT;              /* Fermi-Dirac temperature (eV)                                   */
    double n_electrons;     /* electron count for the chemical potential                      */
    double breakdown_tol;   /* stop when beta <= tol * ||H u_n||_2 (default 1e-12)           */
    double mu_tol;          /* bisection stops when the bracket is narrower (default 1e-13)  */
    int    nu;              /* Krylov dimension (<= 64)                                       */
    int    max_bisect;      /* bisection step limit (default 100)                             */
    int    two_pass;        /* 1: memory-saving workflow of Eq. 3 (G computed twice)         */
    int    n_classes;       /* 0..4 size classes for nu                                       */
    int    class_max_atoms[4];
    int    class_nu[4];
    int    max_neighbors;   /* capacity of a neighbour row (0: default 64)                    */
    int    max_cluster;     /* capacity of a cluster (0: default 512)                         */
    int    schedule;        /* 0: plain (persistent CTAs, static atom order), 1: batched
                               (persistent CTAs pulling atoms from a cluster-size-sorted queue) */
    int    timing;          /* 1: time the kernels of each call with CUDA events (elses_stats) */
    int    k3_ctas_per_sm;  /* resident Krylov CTAs per SM (0: as many as fit); fewer CTAs keep
                               more of the per-CTA Krylov bases in L2                            */
    int    force_mode;      /* forces of elses_energy_force: 0 = density-matrix adjoint
                               (dF/dH = rho, dF/dS = -rhoE; exact when the Krylov space spans the
                               cluster), 1 = exact gradient of the truncated method
                               (elses_omega_gradient chained with dH/dR, dS/dR)                 */
    int    krylov_block;    /* 0: one Krylov space per column, K_nu(H_C, e_j); 1: one block space
                               per atom J started by its 4 orbitals, K(H_C, [e_4J .. e_4J+3]),
                               of dimension nu (>= 4; the band form of block Arnoldi), shared
                               by the atom's 4 columns (the alternative reading of the multiple
                               Arnoldi method); elses_omega_gradient is not available with it */
    int    batch_atoms;     /* atoms per Krylov -> eigensolver batch (0: automatic, sized by a
                               memory budget); smaller batches need less device memory          */
    int    autotune;        /* 1: elses_build_clusters runs elses_autotune on its first build
                               (ignored when k3_ctas_per_sm is set)                              */
    int    graph;           /* 1: elses_energy_force replays its step as a CUDA graph: the first
                               call with a new launch plan runs as usual, the next captures the
                               device work (columns, the bisection's fixed launch sequence,
                               density, scalars, forces at the device-resident mu), later calls
                               replay it with one host synchronisation; a rebuild that keeps the
                               plan and buffers keeps the graph. Results equal the eager path.   */
    int    k3_lanes;        /* lanes per column of the Krylov kernel: 0 = automatic (a half-warp
                               per column, two columns per warp, for the size classes whose
                               clusters would leave the last slot of 32 atoms at most half full;
                               forces from the density matrix and per-column spaces only),
                               32 = one warp per column always                                   */
    int    max_qr_sweeps;   /* cap on the implicit-shift QR sweeps of one projected eigenproblem
                               (0: 30 nu); a column that needs more sets ELSES_ERR_TIMEOUT       */
    int    reorth;          /* second Gram-Schmidt pass of the per-column spaces: 0 = a second
                               classical pass, h2 = SU^T w (CGS2); 1 = its coefficients from the
                               projected overlap already formed, h2 = -(S' - I) h1 (equal to
                               SU^T (w - U h1) in exact arithmetic), so that both passes
                               subtract U (h1 + h2) in one sweep of the basis. The two spaces
                               agree to rounding; the results follow S' and H' formed from the
                               basis itself, so they agree to rounding too, and so does the
                               exact gradient (it differentiates the recursion in exact
                               arithmetic, where the second pass vanishes). Block spaces
                               (krylov_block) always use 0.                                    */
    int    keep_factors;    /* several batches (batch_atoms < N) in the stored workflow: where the
                               density (or G(z), the spectra on the pattern, the exact gradient)
                               later needs V of every column, keep each batch's eigen-factors --
                               the Householder reflectors and L packed (nu_max (nu_max + 1)
                               doubles per column), the recorded Givens rotations in a pool
                               shared by all columns (17 bytes each, about nu^2 per column) --
                               instead of forming V per batch: 0 = never (V per batch), 1 = a
                               pool of at most 60% of the free device memory at the build (V per
                               batch when that holds fewer than nu_max^2 / 2 rotations per
                               column), n >= 2 = a pool of n rotations per column. A column
                               whose rotations do not fit gets V formed instead. Results equal
                               those of V formed per batch to rounding, and those of one batch
                               exactly. A pass over every column starts the pool afresh. The
                               pool is memory the build takes for the system's lifetime: about
                               3x that of V at nu = 30 (the 10^6-atom system: 100 GB for 31 GB). */
} elses_params;

/* Counters and event timings of the calls since the last build (timing = 1 for the times). */
typedef struct elses_stats {
    long long launches;     /* kernels launched                                              */
    long long columns;      /* columns solved (a3-a6)                                        */
    long long krylov_launches;
    int bisect_steps;       /* steps of the last bisection                                   */
    int k3_ctas_per_sm;     /* resident Krylov CTAs per SM of the launch shape in use          */
    double t_krylov_ms;     /* Krylov build + projection kernels (a3, a4)                    */
    double t_eig_ms;        /* projected eigenproblem kernels (a5, a6)                       */
    double t_bisect_ms;     /* bisection and scalar reductions (a7, a9)                      */
    double t_density_ms;    /* density-matrix kernels (a8)                                   */
    double t_force_ms;      /* force kernels (a10)                                           */
    double krylov_flops;    /* algorithmic FP64 flops of the Krylov kernels (a3, a4): per column
                               nu_eff sparse products with H and with S of the same vector, formed
                               together (per off-site block: 43 flops in the two-centre form of
                               Slater-Koster systems -- the projection t = u . x_p, 5 flops,
                               shared by the H and the S block, 19 each -- 64 for two dense 4x4
                               blocks; on-site H diagonal 4 per atom, on-site S = I none) plus
                               CGS2 and projection sum_{n<nu}(6(n+1)+2) n_c
                               + sum_{n<nu-1}(6(n+1)+4) n_c, n_c = 4 |cluster|; with reorth = 1
                               the second sum is sum_{n<nu-1}((2(n+1)+4) n_c + 2(n+1)^2)     */
    double t_adjoint_ms;    /* exact-gradient kernels (elses_omega_gradient)                  */
    double adjoint_flops;   /* algorithmic FP64 flops of the exact-gradient kernels: per column
                               (nu = nu_eff, n_c, b_off in-cluster blocks applied from the
                               lists, p = 24 flops per two-centre block product or 32 dense, n_at
                               cluster atoms; the n_at terms count the on-site blocks where they
                               act as diagonals, Slater-Koster systems, and are 0 otherwise)
                               8 nu^2 n_c (the products G_U = 2 (HU Hh + SU Sh), Y_H = U Hh,
                               Y_S = U Sh) + 6 nu^3 (the Rayleigh-Ritz gradient)
                               + (nu - 1)(8 n_c + p b_off + 4 n_at) + 5 n_c nu (nu - 1) (the
                               reverse Gram-Schmidt sweep with its H products)
                               + 64 nu (b_off + n_at) (the sampled dH and dS blocks, H and S);
                               plus the krylov_flops formula when the bases are recomputed      */
    long long kept_rotations;   /* rotations in the pool of kept eigen-factors (keep_factors)     */
    long long v_formed_columns; /* columns of the last pass whose V was formed as the pool was full */
    int batches;            /* Krylov -> eigensolver batches of a pass over every column         */
    int keep_factors;       /* 1 when the eigen-factors of every column are kept across batches  */
} elses_stats;

typedef struct elses_system_s* elses_system;

/* a1 + a2: neighbour lists and clusters (periodic cell lists, brute force inside cells), then
 * the Slater-Koster H and S on the pattern. If *sys is NULL a system is created; otherwise the
 * existing system is rebuilt for new positions (same atom count), reusing its memory.
 * pos_dev: double[N][3] device. box_host: double[3] host. sk, params: host structs (copied).
 * Passage: Eq. 1 (sparse symmetric H, S) and the redundant local build of H and S
 * (data-communication saving, item I of the computational issues). */
int elses_build_clusters(elses_system* sys, int n_atoms, const double* pos_dev,
                         const double* box_host, const elses_sk* sk,
                         const elses_params* params, void* stream);

/* Replace H and S by caller values (double[nnzb][4][4] device each, [e][a][b] = X_(I,a),(J,b) for
 * block e = (I, J)), on the system's own pattern (row_ptr_dev = col_idx_dev = NULL; nnzb is then
 * ignored) or on the caller's block pattern: row_ptr_dev int32[N+1], col_idx_dev int32[nnzb]
 * (device), rows strictly ascending, every diagonal block present, the pattern symmetric (block
 * (J, I) present with (I, J)) and no row longer than max_neighbors. The caller's pattern replaces
 * the neighbour pattern until the next elses_build_clusters: it is the pattern of the sparse
 * products inside each column's cluster (the clusters stay those of r_cluster around the
 * positions), of rho and rhoE (elses_density_matrix), of G and of the ICOHP. The on-site blocks
 * are applied as full blocks. The pattern is checked on the host before anything changes
 * (ELSES_ERR_ARG, or ELSES_ERR_CAPACITY for a row over max_neighbors). Forces need the
 * Slater-Koster H and S and are unavailable afterwards (ERR_STATE). Synchronises `stream` when a
 * pattern is given. Passage: Eq. 1 (H and S sparse, real symmetric, S positive definite). */
int elses_set_hs(elses_system sys, int nnzb, const int* row_ptr_dev, const int* col_idx_dev,
                 const double* H_dev, const double* S_dev, void* stream);

/* Autotuner of the Krylov kernel's launch shape (a3, a4). For each cluster size class of the
 * system (clusters up to its capacity in atoms; one CTA per atom, persistent), run = 1 times
 * the kernel at every count of resident CTAs per SM that fits -- fewer CTAs keep more of their
 * Krylov bases in L2, more hide more latency -- on a sample of the class's own atoms (up to two
 * full waves, in launch order), and keeps the fastest per atom. With the work queue
 * (schedule = 1) and at least four atoms per CTA it then times the whole class in both orders
 * of its atoms, decreasing cluster size (a short tail) and atom order (neighbouring clusters in
 * flight together share H and S in L2), and keeps the faster. The choices hold for the later
 * calls of this system and its rebuilds. The timed launches use the column buffers, so columns
 * computed before are invalidated; the results of later calls do not depend on the shape or
 * the order (bit for bit). run = 0 only reports the shapes in use. classes_out: optional host
 * int[3 * max_classes], triples (cluster capacity of the class in atoms, CTAs per SM,
 * queue order: 0 static, 1 by size, 2 by atom), each class once (tuned at the first batch that
 * has it); n_host: the number of classes. ERR_STATE for run = 1 when
 * params.k3_ctas_per_sm fixes the shape. Passage: none (a launch-shape choice). */
int elses_autotune(elses_system sys, int run, int max_classes, int* classes_out, int* n_host,
                   void* stream);

/* a3-a6: per-column Krylov build, projection, projected generalized eigenproblem and spectra
 * for columns [col_begin, col_end) (whole atoms: both multiples of 4). Keeps the spectra (and,
 * unless two_pass, what rho needs). If n_z > 0, also writes G_ij(z) for the pattern rows i of
 * each column j into G_dev[(e*16 + a*4 + b)*n_z + iz][2] (re, im) for block e = (I, J) holding
 * G_(I,a),(J,b), z_host[iz] = (re, im). nu_eff_dev: optional int[M] device output. The columns
 * are computed in the system's batches of atoms (params.batch_atoms): a range that starts
 * inside a batch recomputes it from its first atom (the same columns again; G is written for
 * the range only). With keep_factors and several batches, a range of every column (n_z = 0)
 * starts the pool of kept rotations afresh, and until it returns its columns count as not
 * computed. Passage: Eq. 1 and the generation of G column by column. */
int elses_green_columns(elses_system sys, int col_begin, int col_end, int n_z,
                        const double* z_host, double* G_dev, int* nu_eff_dev, void* stream);

/* a7: chemical potential by bisection on N(mu) = sum_j sum_k 2 f(e_k - mu) d_k c_k over all
 * columns (requires every column). Writes mu and N(mu) to host. Passage: the bisection for mu
 * after the first calculation of G (Eq. 3 and the text after it). */
int elses_find_mu(elses_system sys, double* mu_host, double* n_at_mu_host, void* stream);

/* a8: density matrix rho_(I,a),(J,b) = 2 sum_k f(e_k - mu) Z_(I,a),k c_k of column j = 4J + b
 * and its energy-weighted form, on the pattern (double[nnzb][4][4] device each; rhoE_dev may be
 * NULL). In two_pass mode the columns are recomputed first. Passage: Eq. 2, Eq. 3. */
int elses_density_matrix(elses_system sys, double mu, double* rho_dev, double* rhoE_dev,
                         void* stream);

/* a9 at a given mu: N(mu), E_band = sum 2 f g c = Tr(rho H), Omega and F_free = Omega + mu N_e
 * (host doubles; any may be NULL). Passage: Eq. 6. */
int elses_energies(elses_system sys, double mu, double* n_host, double* e_band_host,
                   double* omega_host, double* f_free_host, void* stream);

/* a3-a10 in one call: columns, mu, rho, energies, forces F_I = -dF_free/dR_I (double[N][3]
 * device; may be NULL). Host outputs may be NULL. Passage: energy and force for MD from rho. */
int elses_energy_force(elses_system sys, double* mu_host, double* e_band_host,
                       double* f_free_host, double* forces_dev, void* stream);

/* a10 alone: forces F_I = -dF_free/dR_I (double[N][3] device) from the rho and rhoE kept by the
 * last elses_energy_force on the current positions (the adjoint dF/dH = rho, dF/dS = -rhoE
 * chained with the Slater-Koster dH/dR, dS/dR), or with force_mode = 1 from the exact gradient
 * of elses_omega_gradient at that call's chemical potential; ERR_STATE if there are none.
 * Asynchronous. */
int elses_forces(elses_system sys, double* forces_dev, void* stream);

/* Exact gradient of Omega = sum_j Omega_j at fixed mu through the truncated Krylov method:
 * dOmega/dH and dOmega/dS with the motion of every column's Krylov space K_nu(H_C, e_j) with H
 * included (Omega_j = sum_k d_k c_k w(e_k), w(e) = -2 kT ln(1 + exp(-(e - mu)/kT)); the paper
 * gives forces from rho alone, the density-matrix adjoint, which this equals only when the
 * Krylov space spans the cluster). Outputs double[nnzb][4][4] device, [e][a][b] =
 * dOmega / dH_(I,a),(J,b) for block e = (I, J) (on-site blocks included), summed over the
 * columns of atoms [atom_begin, atom_end); both are overwritten. The gradient of F_free at fixed
 * N_e is this at the chemical potential. Needs every column computed at the current positions
 * (elses_green_columns over all columns, or elses_energy_force); in the two-pass mode each
 * batch's columns are recomputed first. ERR_ARG for a bad range or null outputs, ERR_STATE
 * without the columns, ERR_NOT_IMPLEMENTED for block spaces (krylov_block = 1). Synchronises
 * `stream` (device status check). */
int elses_omega_gradient(elses_system sys, double mu, int atom_begin, int atom_end, double* dH_dev,
                         double* dS_dev, void* stream);

/* (pi)COHP analysis, Eqs. 4-8: the ICOHP of each block e = (I, J) of the pattern,
 * B_IJ = sum_ab H_(J,b);(I,a) rho_(I,a);(J,b) (the Fermi-weighted energy integral of the COHP of
 * Eq. 4 taken by residues), and its sigma / pi parts from the Slater-Koster split of the off-site
 * H (B = B_sigma + B_pi off-site; on-site blocks have B_sigma = B_pi = 0). sum over all blocks of
 * B equals E_band (Eq. 6). rho_dev: double[nnzb][4][4] from elses_density_matrix. Outputs
 * double[nnzb] device (B_sigma, B_pi may be NULL; they need the Slater-Koster H: ERR_STATE after
 * elses_set_hs). Asynchronous on `stream`. */
int elses_icohp(elses_system sys, const double* rho_dev, double* B_dev, double* Bsig_dev,
                double* Bpi_dev, void* stream);

/* Energy-resolved COHP (Eq. 4) and density of states at the complex energies z_host[n_z][2]
 * (z = e + i eta, eta > 0: each pole's delta function of Im G(e + i0) becomes a Lorentzian of
 * half-width eta): C_IJ(z) = -(1/pi) Im sum_ab H_(J,b);(I,a) G_(I,a);(J,b)(z) per block e = (I, J)
 * of the pattern, with G from the poles and residues of the columns (elses_green_columns), its
 * sigma and pi parts as in elses_icohp (off-site only), and DOS(z) = -(1/pi) Im Tr(G(z) S)
 * = -(1/pi) Im sum_j sum_k d_k c_k / (z - e_k). Outputs: device double[nnzb][n_z] (C, C_sigma,
 * C_pi; any may be NULL; sigma / pi need the Slater-Koster H) and host double[n_z] (dos, may be
 * NULL). Needs every column computed; in the two-pass mode the batches are recomputed. Summed
 * over blocks, C(z) is -(1/pi) Im sum_j sum_k g_k c_k / (z - e_k), the band-energy spectrum.
 * Synchronises `stream`. */
int elses_cohp_spectrum(elses_system sys, int n_z, const double* z_host, double* C_dev,
                        double* Csig_dev, double* Cpi_dev, double* dos_host, void* stream);

/* Copy-out accessors: each copies library data into caller-owned device buffers (any of which
 * may be NULL to skip it) on `stream`; sizes are returned through the host pointers first
 * (call once with NULL buffers to learn them). */
int elses_get_pattern(elses_system sys, int* nnzb_host, int* row_ptr_dev, int* col_idx_dev,
                      void* stream);                               /* int[N+1], int[nnzb]       */
int elses_get_hs(elses_system sys, double* H_dev, double* S_dev, void* stream);
                                                                   /* double[nnzb][4][4] each   */
int elses_get_clusters(elses_system sys, long long* total_host, int* max_cluster_host,
                       int* cl_ptr_dev, int* cl_idx_dev, void* stream);
              /* int[N+1], int[total]; with r_cluster <= 0 every cluster is the whole system and
                 only the sizes are returned                                                   */
int elses_get_spectra(elses_system sys, int* nu_max_host, double* eps_dev, double* c_dev,
                      double* d_dev, double* g_dev, int* nu_eff_dev, void* stream);
              /* double[M][nu_max] each (entries k >= nu_eff[j] are zero), int[M]              */
/* Counters and timings accumulated since the last build or elses_reset_stats. */
int elses_get_stats(elses_system sys, elses_stats* stats_host);
int elses_reset_stats(elses_system sys);

/* Measurement utility (not part of the method): FP64 fused multiply-add throughput of the
 * current device in GFLOP/s (2 flops per FMA), from a kernel of independent FMA chains on
 * every SM, timed with CUDA events. */
int elses_probe_fp64(double* gflops_host, void* stream);

/* Allocation-free chemical-potential bisection. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need mu -- an application
 * whose own allocator has already reserved the device memory, or a loop in which allocation
 * (and the synchronisation it implies) is not allowed. It runs the bisection kernels of
 * elses_find_mu without their kept-pole window (every pole is summed at every step, in another
 * order), so mu agrees with elses_find_mu to rounding (a few 1e-13 eV), on caller-owned spectra
 * in the layout of
 * elses_get_spectra: eps, c, d, g double[n_columns][nu_max] and nu_eff int[n_columns] on the
 * device (g may be NULL unless e_band_host is requested); mu_tol <= 0 and max_bisect <= 0 take
 * the defaults 1e-13 and 100. It calls no cudaMalloc / cudaFree: its scratch (block partial sums,
 * bracket state, ticket) is one static device array of 4096 x 4 + 32 doubles (about 131 KB)
 * that every GPU loading the library holds until exit; a device that would need more than
 * 4096 reduction blocks is rejected with ELSES_ERR_CAPACITY. Every call looks the array's
 * address up on the current device (nothing is cached, so a context re-created after
 * cudaDeviceReset is followed); the first call on a device may load the library's device code,
 * so make that first call before any stream capture. All calls share the
 * array and it keeps the last call's contents: calls that overlap on the GPU race and must be
 * serialised by the caller. Synchronises `stream` before returning. */
int elses_find_mu_static(int n_columns, int nu_max, const double* eps_dev, const double* c_dev,
                         const double* d_dev, const double* g_dev, const int* nu_eff_dev,
                         double kT, double n_electrons, double mu_tol, int max_bisect,
                         double* mu_host, double* n_at_mu_host, double* e_band_host,
                         void* stream);

void elses_system_destroy(elses_system sys);
const char* elses_last_error(void);
int elses_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ELSES_H */
