// Host runtime of the C ABI (include/elses.h): system handle, memory, launch sequencing.
//
// Order of one energy + force evaluation (the memory-saving workflow of Eq. 3 when two_pass,
// otherwise the per-column quantities of the first pass are kept and reused):
//   build_clusters : cells -> neighbour CSR -> cluster CSR -> Slater-Koster H, S   (a1, a2)
//   green_columns  : batches of atoms: Krylov build + projection (one CTA per atom), then the
//                    projected eigenproblem (one thread per column)                  (a3-a6)
//   find_mu        : device-resident bisection, one launch per step                  (a7)
//   density_matrix : rho, rhoE on the pattern                                        (a8)
//   energies       : N, E_band, Omega, F_free                                        (a9)
//   forces         : per-block gradient contraction, per-atom sums                   (a10)
// The autotuner (autotune.cu) and the CUDA-graph form of the step (graph.cu) share the state and
// helpers declared in system_impl.h.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "system_impl.h"

using namespace elses;

static thread_local std::string g_err;

namespace elses {
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int report_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
}  // namespace elses

unsigned long long g_alloc_epoch = 0;

namespace elses {

int nu_of_params(const elses_params& p) {
    int m = p.nu;
    for (int c = 0; c < p.n_classes; ++c) m = std::max(m, p.class_nu[c]);
    return m;
}

int check_status(elses_system s, cudaStream_t st, bool allow_breakdown_warning) {
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, s->counters.p + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());
    s->collect();
    if (h & DEV_CAPACITY) return fail(ELSES_ERR_CAPACITY, "a neighbour or cluster list exceeded its capacity");
    if (h & DEV_NOT_SPD) return fail(ELSES_ERR_NOT_SPD, "projected overlap S' is not positive definite");
    if (h & DEV_NONFINITE) return fail(ELSES_ERR_NONFINITE, "non-finite value in the Krylov build");
    if (h & DEV_TIMEOUT) return fail(ELSES_ERR_TIMEOUT, "projected eigensolver did not converge");
    if (h & DEV_ARG) return fail(ELSES_ERR_ARG, "invalid device-side argument");
    if ((h & DEV_BREAKDOWN) && allow_breakdown_warning) return ELSES_WARN_BREAKDOWN;
    return ELSES_OK;
}

int clear_status(elses_system s, cudaStream_t st) {
    CUDA_TRY(cudaMemsetAsync(s->counters.p + 2, 0, sizeof(int), st));
    return 0;
}

// Column storage, Krylov launch shape and batch buffers for the current sizes.
int prepare_columns(elses_system s) {
    s->nu_max = nu_of_params(s->p);
    s->na_max = ((s->max_cl + 31) / 32) * 32;
    const int nm = s->nu_max;
    // list capacity per position: in-cluster neighbours, the on-site block excluded when it
    // is applied as a diagonal (Slater-Koster systems)
    s->deg_cap = s->user_hs ? s->max_nb : std::max(1, s->max_nb - 1);
    int dev = 0;
    cudaGetDevice(&dev);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int kdeg = s->user_hs ? s->max_nb : s->deg_cap;
    if ((int)krylov_smem_bytes(s->na_max, kdeg) > smem_optin)
        return fail(ELSES_ERR_CAPACITY, "cluster of %d atoms needs %zu B of shared memory (max %d)",
                    s->max_cl, krylov_smem_bytes(s->na_max, kdeg), smem_optin);
    if ((long long)eig_smem_max(nm) > smem_optin)
        return fail(ELSES_ERR_CAPACITY, "Krylov dimension %d needs %zu B of shared memory in the eigensolver (max %d)",
                    nm, eig_smem_max(nm), smem_optin);
    // batch of atoms for the Krylov -> eigensolver hand-off
    {
        const size_t PK0 = (size_t)nm * (nm + 1) / 2;
        const size_t per_col0 = sizeof(double) * (2 * PK0 + 3 * (size_t)nm + eig_tri_doubles(nm) + eig_fac_doubles(nm) +
                                                  2 * eig_rot_cap(nm)) + eig_rot_cap(nm) + sizeof(int) * (nm + 1);
        // batch buffers: up to 16 GB or a fifth of the free memory, so that large systems run in a
        // few long launches (shorter Krylov launch tails; measured on 10^6 atoms: 4800-atom
        // batches 17.7 s per step, 37000-atom batches 17.3 s) and systems of a few 10^4 atoms in
        // one batch, which needs no V for the energy (the 32768-atom composite: 2 batches at 8 GB)
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const size_t budget = std::max<size_t>(size_t(1) << 30, std::min<size_t>(size_t(16) << 30, free_b / 5));
        const size_t cols0 = std::max<size_t>(128, budget / per_col0);
        s->batch_atoms = (int)std::min<size_t>((size_t)s->n, std::max<size_t>(32, cols0 / 4));
        if (s->p.batch_atoms > 0) s->batch_atoms = std::min(s->n, s->p.batch_atoms);
    }
    // size classes: atoms grouped by cluster slots, largest class first; inside a class the
    // batched form orders atoms by decreasing cluster size (or atom order, as tuned), the plain
    // form by index. Where two columns per warp apply (forces from the density matrix, one space
    // per column, k3_lanes != 32) the slots hold 16 atoms: a class of an odd number c of them
    // runs k_krylov_half (one column per half-warp, capacity 16 c) when it keeps at least as many
    // warps per SM as k_krylov at capacity 16 (c + 1), or as the autotuner chose; the others run
    // k_krylov. Otherwise slots of 32.
    const bool half_ok = s->p.k3_lanes != 32 && s->p.force_mode == 0 && !s->p.krylov_block;
    const int gslot = half_ok ? 16 : 32;
    std::vector<int> ord;
    ord.reserve(s->n);
    s->k3_launches.clear();
    size_t scratch = 0;
    int best_items = -1;
    // an odd 16-slot class runs with half-warps, or with whole warps inside the next (even) class
    auto odd_half = [&](int k) {
        const int th = k < (int)s->tuned_half.size() ? s->tuned_half[k] : 0;
        if (th) return th == 1;
        return krylov_half_blocks_per_sm(16 * k, kdeg) >= 2 * krylov_blocks_per_sm(16 * (k + 1), kdeg);
    };
    for (int b = 0; b < s->n; b += s->batch_atoms) {
        const int e = std::min(s->n, b + s->batch_atoms);
        size_t batch_off = 0;
        for (int ns = s->na_max / gslot; ns >= 1; --ns) {
            const int key = gslot * ns / 16;
            const bool half = half_ok && (ns & 1) && odd_half(key);
            if (half_ok && (ns & 1) && !half) continue;          // merged into class ns + 1
            const bool merge_below = half_ok && !(ns & 1) && ns > 1 && !odd_half(key - 1);
            const int begin = (int)ord.size();
            for (int a = b; a < e; ++a) {
                const int c = (s->h_clsize[a] + gslot - 1) / gslot;
                if (c == ns || (merge_below && c == ns - 1)) ord.push_back(a);
            }
            const int count = (int)ord.size() - begin;
            if (count == 0) continue;
            const int na = gslot * ns;
            const bool by_atom = key < (int)s->tuned_order.size() && s->tuned_order[key] == 2;
            if (s->p.schedule == 1 && !by_atom)
                std::stable_sort(ord.begin() + begin, ord.end(),
                                 [&](int x, int y) { return s->h_clsize[x] > s->h_clsize[y]; });
            int bps = s->p.krylov_block ? block_krylov_blocks_per_sm(na, kdeg)
                      : half             ? krylov_half_blocks_per_sm(na, kdeg)
                                         : krylov_blocks_per_sm(na, kdeg);
            if (bps < 1) return fail(ELSES_ERR_CAPACITY, "Krylov kernel cannot be resident (%d-atom class)", na);
            // a count fixed by the caller or chosen by the autotuner may use the 4-CTA form
            const int bps_max = (s->p.krylov_block || half) ? bps : krylov_blocks_per_sm_max(na, kdeg);
            if (s->p.k3_ctas_per_sm > 0) bps = std::min(bps_max, s->p.k3_ctas_per_sm);
            else if (key < (int)s->tuned_bps.size() && s->tuned_bps[key] > 0) bps = std::min(bps_max, s->tuned_bps[key]);
            const int grid = std::min(count, s->num_sms * bps);
            s->k3_launches.push_back({b, e, begin, count, na, grid, bps, half ? 1 : 0, key, batch_off});
            batch_off += s->p.krylov_block ? (size_t)grid * block_krylov_scratch_doubles(nm, na)
                                           : (size_t)grid * kWarpsPerAtom * 2 * nm * na * 4;
            scratch = std::max(scratch, batch_off);
            if (count > best_items) { best_items = count; s->k3_bps = bps; }
        }
    }
    TRY(s->order.ensure(s->n));
    CUDA_TRY(cudaMemcpy(s->order.p, ord.data(), sizeof(int) * s->n, cudaMemcpyHostToDevice));
    TRY(s->kscratch.ensure(scratch));
    // batch of atoms for the Krylov -> eigensolver hand-off
    const size_t PK = (size_t)nm * (nm + 1) / 2;
    const size_t bc = 4 * (size_t)s->batch_atoms;
    const size_t bc_pad = ((bc + 31) / 32) * 32;
    TRY(s->Hp.ensure(bc * PK));
    TRY(s->Sp.ensure(bc * PK));
    TRY(s->urow.ensure(bc * nm));
    TRY(s->surow.ensure(bc * nm));
    TRY(s->hurow.ensure(bc * nm));
    (void)bc_pad;
    TRY(s->etri.ensure(bc * eig_tri_doubles(nm)));
    TRY(s->efac.ensure(bc * eig_fac_doubles(nm)));
    TRY(s->erot_c.ensure(bc * eig_rot_cap(nm)));
    TRY(s->erot_s.ensure(bc * eig_rot_cap(nm)));
    TRY(s->erot_k.ensure(bc * eig_rot_cap(nm)));
    TRY(s->erot_n.ensure(bc));
    TRY(s->ewt.ensure(bc * 2 * nm));
    TRY(s->eperm.ensure(bc * nm));
    const size_t M = s->M;
    TRY(s->eps.ensure(M * nm));
    TRY(s->cc.ensure(M * nm));
    TRY(s->dd.ensure(M * nm));
    TRY(s->gg.ensure(M * nm));
    TRY(s->nu_eff.ensure(M));
    if (!s->p.two_pass) {
        TRY(s->V.ensure(M * nm * nm));
        TRY(s->UP.ensure((size_t)s->nnzb * 16 * nm));
    } else {
        int maxblk = 0;
        for (int b = 0; b < s->n; b += s->batch_atoms) {
            const int e = std::min(s->n, b + s->batch_atoms);
            maxblk = std::max(maxblk, s->h_row_ptr[e] - s->h_row_ptr[b]);
        }
        TRY(s->Vb.ensure(bc * nm * nm));
        TRY(s->UPb.ensure((size_t)maxblk * 16 * nm));
    }
    TRY(s->rho.ensure((size_t)s->nnzb * 16));
    TRY(s->rhoE.ensure((size_t)s->nnzb * 16));
    // exact forces in the stored workflow: the Krylov pass keeps every column's bases (when they
    // fit in 48 GB) so that the adjoint does not recompute them
    s->use_store = false;
    if (s->p.force_mode == 1 && !s->p.two_pass && !s->p.krylov_block) {
        s->bvec = (size_t)nm * s->na_max * 4;
        s->bstride = (3 * s->bvec + (size_t)nm * nm + (size_t)nm * (nm + 1) / 2 + 3) & ~(size_t)3;
        const size_t need = M * s->bstride;
        if (need * sizeof(double) <= (size_t(48) << 30)) {
            TRY(s->bstore.ensure(need));
            s->use_store = true;
        }
    }
    // several batches in the stored workflow, keep_factors set: the eigen-factors of every column
    // are kept (a pool of rotations of at most 60% of the free memory, or keep_factors per
    // column) so that V need not be formed per batch; too small a pool does not pay, and V is
    // formed per batch then
    const bool arch_was = s->arch;
    s->arch = false;
    if (!s->p.two_pass && s->batch_atoms < s->n && s->p.keep_factors > 0) {
        const size_t fixed = M * (sizeof(double) * (eig_arch_fac_doubles(nm) + 2 * (size_t)nm) +
                                  sizeof(int) * ((size_t)nm + 1) + sizeof(unsigned long long)) + bc * sizeof(int);
        const size_t per_rot = 2 * sizeof(double) + 1;
        size_t cap = 0;
        if (s->p.keep_factors > 1) {
            cap = M * (size_t)s->p.keep_factors;
        } else if (arch_was && s->arch_M == M && s->arch_nm == nm) {
            cap = s->arch_cap;   // a rebuild of the same size keeps the pool it planned
        } else {
            // the archive a previous build planned counts as free (a rebuild keeps its plan)
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            free_b += sizeof(double) * (s->afac.cap + s->arot_c.cap + s->arot_s.cap + s->ewt_all.cap) +
                      s->arot_k.cap + sizeof(int) * (s->aperm.cap + s->an.cap + s->alist.cap) +
                      sizeof(unsigned long long) * (s->aoff.cap + s->acnt.cap);
            const size_t avail = free_b / 10 * 6;
            cap = avail > fixed ? (avail - fixed) / per_rot : 0;
            cap = std::min(cap, M * eig_rot_cap(nm));
            if (cap < M * (size_t)nm * nm / 2) cap = 0;
        }
        if (cap > 0) {
            const unsigned long long epoch = g_alloc_epoch;
            TRY(s->afac.ensure(M * eig_arch_fac_doubles(nm)));
            TRY(s->aperm.ensure(M * nm));
            TRY(s->an.ensure(M));
            TRY(s->aoff.ensure(M));
            TRY(s->arot_c.ensure(cap));
            TRY(s->arot_s.ensure(cap));
            TRY(s->arot_k.ensure(cap));
            TRY(s->acnt.ensure(3));
            TRY(s->alist.ensure(bc));
            TRY(s->ewt_all.ensure(M * 2 * nm));
            if (epoch != g_alloc_epoch || !s->arch_init) {   // new buffers: no column kept yet
                CUDA_TRY(cudaMemset(s->acnt.p, 0, 3 * sizeof(unsigned long long)));
                CUDA_TRY(cudaMemset(s->an.p, 0xff, s->an.cap * sizeof(int)));
                s->arch_init = true;
            }
            s->arch = true;
            s->arch_cap = cap;
            s->arch_M = M;
            s->arch_nm = nm;
        }
    }
    if (!s->arch) {
        s->arch_init = false;
        s->arch_cap = 0;
        s->afac.release();
        s->aperm.release();
        s->an.release();
        s->aoff.release();
        s->arot_c.release();
        s->arot_s.release();
        s->arot_k.release();
        s->acnt.release();
        s->alist.release();
        s->ewt_all.release();
    }
    TRY(s->gblock.ensure((size_t)s->nnzb * 3));
    TRY(s->partials.ensure(4 * (size_t)reduce_grid()));
    TRY(s->act.ensure(M * nm));
    TRY(s->act_n.ensure(reduce_grid()));
    TRY(s->act_below.ensure(reduce_grid()));
    TRY(s->bstate.ensure(1));
    TRY(s->ticket.ensure(1));
    CUDA_TRY(cudaMemset(s->ticket.p, 0, sizeof(unsigned)));
    s->atom_done.assign(s->n, 0);
    s->atoms_done = 0;
    s->have_mu = false;
    s->have_rho = false;
    s->v_lazy = false;
    s->v_arch = false;
    return 0;
}

// A pass over every column in the archive's form: the pool starts empty, and until a batch is
// done its columns count as not computed (a pass that stops early leaves them so).
int reset_archive(elses_system s, cudaStream_t st) {
    CUDA_TRY(cudaMemsetAsync(s->acnt.p, 0, 2 * sizeof(unsigned long long), st));
    s->atom_done.assign(s->n, 0);
    s->atoms_done = 0;
    s->v_arch = false;
    return 0;
}

// The second stream: work launched on it after fork_side runs beside `st` until join_side.
int fork_side(elses_system s, cudaStream_t st) {
    if (!s->side) {
        CUDA_TRY(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
    }
    CUDA_TRY(cudaEventRecord(s->ev_fork, st));
    CUDA_TRY(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
    return 0;
}
int join_side(elses_system s, cudaStream_t st) {
    CUDA_TRY(cudaEventRecord(s->ev_join, s->side));
    CUDA_TRY(cudaStreamWaitEvent(st, s->ev_join, 0));
    return 0;
}

// Krylov-kernel arguments for atoms [b, e) (the launch fields are set per size class).
KrylovArgs krylov_args(elses_system s, int b, int e) {
    const int nm = s->nu_max;
    KrylovArgs ka{};
    ka.n_atoms = s->n;
    ka.row_ptr = s->row_ptr.p;
    ka.col_idx = s->col_idx.p;
    ka.H = s->H.p;
    ka.S = s->S.p;
    ka.skr = s->user_hs ? nullptr : s->skr.p;   // structured two-centre products for SK systems
    ka.cl_ptr = s->p.r_cluster > 0 ? s->cl_ptr.p : nullptr;
    ka.cl_idx = s->p.r_cluster > 0 ? s->cl_idx.p : nullptr;
    ka.atom_begin = b;
    ka.atom_end = e;
    ka.nu_max = nm;
    ka.nu_default = s->p.nu;
    ka.n_classes = s->p.n_classes;
    for (int c = 0; c < 4; ++c) {
        ka.class_max_atoms[c] = s->p.class_max_atoms[c];
        ka.class_nu[c] = s->p.class_nu[c];
    }
    ka.breakdown_tol = s->p.breakdown_tol;
    ka.reorth = s->p.krylov_block ? 0 : s->p.reorth;   // the block build has its own passes
    ka.onsite_diag = s->user_hs ? 0 : 1;   // Slater-Koster on-site blocks: S = I, H diagonal
    ka.deg_max = s->user_hs ? s->max_nb : s->deg_cap;
    ka.scratch = s->kscratch.p;
    ka.Hp = s->Hp.p;
    ka.Sp = s->Sp.p;
    ka.urow = s->urow.p;
    ka.surow = s->surow.p;
    ka.hurow = s->hurow.p;
    ka.nu_eff = s->nu_eff.p;
    ka.status = s->counters.p + 2;
    ka.flops = s->flops_ctr.p;
    ka.bstore = s->use_store ? s->bstore.p : nullptr;
    ka.bstride = s->bstride;
    ka.bvec = s->bvec;
    return ka;
}

// Eigenproblem arguments for atoms [b, e), V written at V.
EigArgs eig_args(elses_system s, int b, int e, double* V) {
    EigArgs ea{};
    ea.ncols = 4 * (e - b);
    ea.col0 = 4 * b;
    ea.nu_max = s->nu_max;
    ea.Hp = s->Hp.p;
    ea.Sp = s->Sp.p;
    ea.urow = s->urow.p;
    ea.surow = s->surow.p;
    ea.hurow = s->hurow.p;
    ea.nu_eff = s->nu_eff.p;
    ea.tri = s->etri.p;
    ea.fac = s->efac.p;
    ea.rot_c = s->erot_c.p;
    ea.rot_s = s->erot_s.p;
    ea.rot_k = s->erot_k.p;
    ea.rot_n = s->erot_n.p;
    ea.perm = s->eperm.p;
    ea.eps = s->eps.p;
    ea.c = s->cc.p;
    ea.d = s->dd.p;
    ea.g = s->gg.p;
    ea.V = V;
    ea.status = s->counters.p + 2;
    ea.max_sweeps = s->p.max_qr_sweeps;   // 0: 30 nu of the column
    if (s->arch) {
        ea.ar.fac = s->afac.p;
        ea.ar.perm = s->aperm.p;
        ea.ar.n = s->an.p;
        ea.ar.off = s->aoff.p;
        ea.ar.rot_c = s->arot_c.p;
        ea.ar.rot_s = s->arot_s.p;
        ea.ar.rot_k = s->arot_k.p;
        ea.ar.cap = s->arch_cap;
        ea.ar.cnt = s->acnt.p;
        ea.ar.list = s->alist.p;
    }
    return ea;
}

// The stored V of every column, from the kept factors, where the energy pass left it unformed
// (G(z), the spectra on the pattern and the adjoint need V itself).
int ensure_V(elses_system s, cudaStream_t st) {
    if (s->v_lazy) {
        s->tic(T_EIG, st);
        eig_vectors(eig_args(s, 0, s->n, s->V.p), st);
        s->toc(st);
        s->stats.launches++;
        s->v_lazy = false;
    }
    if (s->v_arch) {
        s->tic(T_EIG, st);
        eig_vectors_archived(eig_args(s, 0, s->n, s->V.p), st);
        s->toc(st);
        s->stats.launches++;
        s->v_arch = false;
    }
    return 0;
}

// Krylov build + projected eigenproblem for atoms [b, e). Writes V and UP either to the stored
// arrays or to the batch buffers (two-pass), returning the pointers used. form_v false leaves V
// unformed; in the stored workflow that holds for a batch of every atom (its factors then stay in
// the batch buffers until ensure_V or the next batch) and, where the archive is planned, for each
// of several batches (its factors go to the archive); other batches form V.
int run_batch(elses_system s, int b, int e, bool stored, double** V_out, int* v_col0,
              double** UP_out, int* up_block0, cudaStream_t st, bool need_rows, bool form_v) {
    const int nm = s->nu_max;
    std::vector<const elses_system_s::K3Launch*> ls;   // the batch's Krylov launches
    for (const auto& L : s->k3_launches)
        if (L.batch_begin == b) ls.push_back(&L);
    if (ls.empty() || e > ls[0]->batch_end)
        return fail(ELSES_ERR_STATE, "atoms [%d, %d) are not the start of a planned batch", b, e);
    const bool multi = b != 0 || e != s->n;
    const bool keep = stored && !form_v && multi && s->arch;
    if (stored && !form_v && multi && !keep) form_v = true;
    // the batch buffers are about to be overwritten: V of the columns whose factors are there
    // first (the archive's stay where they are)
    if (stored && multi && s->v_lazy) TRY(ensure_V(s, st));
    if (stored) s->v_lazy = false;
    KrylovArgs ka = krylov_args(s, b, e);
    if (stored) {
        ka.UP = s->UP.p;
        ka.up_block0 = 0;
    } else {
        ka.UP = s->UPb.p;
        ka.up_block0 = s->h_row_ptr[b];
    }
    if (!need_rows) ka.UP = nullptr;
    s->tic(T_KRYLOV, st);
    // batched form: the class with the most atoms runs on the caller's stream and the others
    // (few atoms each, partial waves) beside it, one after another, on a second stream
    const bool conc = s->p.schedule == 1 && ls.size() >= 2;
    size_t main_cls = 0;
    for (size_t i = 1; i < ls.size(); ++i)
        if (ls[i]->item_count > ls[main_cls]->item_count) main_cls = i;
    if (conc) TRY(fork_side(s, st));
    for (size_t i = 0; i < ls.size(); ++i) {
        const auto& L = *ls[i];
        cudaStream_t lst = (conc && i != main_cls) ? s->side : st;
        ka.na_max = L.na;
        ka.half = L.half;
        ka.order = s->order.p + L.item_begin;
        ka.n_items = L.item_count;
        ka.scratch = s->kscratch.p + L.scratch_off;
        ka.queue = nullptr;
        if (s->p.schedule == 1) {
            // batched form: persistent CTAs pull atoms from the size-sorted queue
            int* q = s->counters.p + kQueue0 + (int)std::min<size_t>(i, kCounters - kQueue0 - 1);
            CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(int), lst));
            ka.queue = q;
        }
        if (s->p.krylov_block) block_krylov_columns(ka, L.grid, lst);
        else krylov_columns(ka, L.grid, L.bps, lst);
        s->stats.launches++;
        s->stats.krylov_launches++;
    }
    if (conc) TRY(join_side(s, st));
    s->toc(st);

    EigArgs ea = eig_args(s, b, e, stored ? s->V.p + (size_t)4 * b * nm * nm : s->Vb.p);
    s->tic(T_EIG, st);
    projected_eig(ea, st, form_v);
    if (keep) {
        eig_archive(ea, st);
        s->stats.launches += 2;
        s->v_arch = true;
    } else if (stored && s->v_arch) {
        // V formed for these columns: the archive's entries give way
        CUDA_TRY(cudaMemsetAsync(s->an.p + 4 * (size_t)b, 0xff, sizeof(int) * 4 * (size_t)(e - b), st));
    }
    s->toc(st);
    s->stats.launches += 3;
    if (stored && !form_v && !keep) s->v_lazy = true;
    s->stats.columns += 4LL * (e - b);
    *V_out = ea.V;
    *v_col0 = 4 * b;
    *UP_out = ka.UP;
    *up_block0 = ka.up_block0;
    return 0;
}

// Exact dOmega/dH and s_scale * dOmega/dS at mu of the columns of atoms [lo, hi) into gH, gS
// ([nnzb][16], overwritten): per batch, the adjoint kernel per size class, after the batch's
// Krylov columns are recomputed when V is not kept (two-pass mode).
int adjoint_impl(elses_system s, double mu, int lo, int hi, double* gH, double* gS, double s_scale,
                 cudaStream_t st, const double* mu_dev) {
    const int nm = s->nu_max;
    const int kdeg = s->user_hs ? s->max_nb : s->deg_cap;
    TRY(s->adj_acc.ensure(4 * 16 * (size_t)s->nnzb));
    CUDA_TRY(cudaMemsetAsync(s->adj_acc.p, 0, sizeof(unsigned long long) * 4 * 16 * (size_t)s->nnzb, st));
    // launch shapes and scratch: the Krylov kernel's size classes, the adjoint's own residency
    if ((int)s->adj_bps.size() != s->na_max / 32 + 1) s->adj_bps.assign(s->na_max / 32 + 1, 0);
    size_t need = 0;
    std::vector<int> grid(s->k3_launches.size(), 0);
    std::vector<size_t> off(s->k3_launches.size(), 0);
    for (size_t i = 0, used = 0; i < s->k3_launches.size(); ++i) {
        const auto& L = s->k3_launches[i];
        const int na = (L.na + 31) / 32 * 32;   // the adjoint keeps one warp per column
        int& bps = s->adj_bps[na / 32];
        if (bps == 0) bps = adjoint_blocks_per_sm(na, kdeg);
        if (bps < 1) return fail(ELSES_ERR_CAPACITY, "adjoint kernel cannot be resident (%d-atom class)", na);
        grid[i] = std::min(L.item_count, s->num_sms * bps);
        if (i == 0 || L.batch_begin != s->k3_launches[i - 1].batch_begin) used = 0;
        off[i] = used;     // the class launches of a batch run at the same time: own scratch each
        used += (size_t)grid[i] * kWarpsPerAtom * adjoint_warp_doubles(nm, na);
        need = std::max(need, used);
    }
    TRY(s->ascratch.ensure(need));
    if (!s->p.two_pass) TRY(ensure_V(s, st));
    for (int b = 0; b < s->n; b += s->batch_atoms) {
        const int e = std::min(s->n, b + s->batch_atoms);
        if (e <= lo || b >= hi) continue;
        AdjointArgs ga{};
        ga.V = s->V.p;
        ga.v_col0 = 0;
        if (s->p.two_pass) {
            double *Vb = nullptr, *UPb = nullptr;
            int c0 = 0, ub0 = 0;
            TRY(run_batch(s, b, e, false, &Vb, &c0, &UPb, &ub0, st, false));
            ga.V = Vb;
            ga.v_col0 = c0;
        }
        ga.eps = s->eps.p;
        ga.c = s->cc.p;
        ga.d = s->dd.p;
        ga.mu = mu;
        ga.mu_dev = mu_dev;
        ga.kT = s->p.kT;
        ga.acc = s->adj_acc.p;
        ga.nnzb = s->nnzb;
        ga.flops = s->flops_ctr.p + 1;
        ga.status = s->counters.p + 2;
        ga.scratch = s->ascratch.p;
        ga.atom_lo = lo;
        ga.atom_hi = hi;
        ga.bstore = s->use_store ? s->bstore.p : nullptr;
        ga.bstride = s->bstride;
        ga.bvec = s->bvec;
        KrylovArgs ka = krylov_args(s, b, e);
        ka.flops = nullptr;
        ka.UP = nullptr;
        s->tic(T_ADJOINT, st);
        std::vector<size_t> li;
        for (size_t i = 0; i < s->k3_launches.size(); ++i)
            if (s->k3_launches[i].batch_begin == b) li.push_back(i);
        const bool conc = li.size() >= 2;   // the main class beside the others, as for the Krylov pass
        size_t main_cls = 0;
        for (size_t t = 1; t < li.size(); ++t)
            if (s->k3_launches[li[t]].item_count > s->k3_launches[li[main_cls]].item_count) main_cls = t;
        if (conc) TRY(fork_side(s, st));
        for (size_t t = 0; t < li.size(); ++t) {
            const size_t i = li[t];
            const auto& L = s->k3_launches[i];
            cudaStream_t lst = (conc && t != main_cls) ? s->side : st;
            ka.na_max = (L.na + 31) / 32 * 32;
            ka.half = 0;
            ka.order = s->order.p + L.item_begin;
            ka.n_items = L.item_count;
            int* q = s->counters.p + kQueue0 + (int)std::min<size_t>(t, kCounters - kQueue0 - 1);
            CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(int), lst));
            ka.queue = q;
            AdjointArgs gl = ga;
            gl.scratch = s->ascratch.p + off[i];
            adjoint_columns(ka, gl, grid[i], lst);
            s->stats.launches++;
        }
        if (conc) TRY(join_side(s, st));
        s->toc(st);
    }
    s->tic(T_ADJOINT, st);
    adjoint_finish(s->adj_acc.p, 16 * (size_t)s->nnzb, s_scale, gH, gS, st);
    s->toc(st);
    s->stats.launches++;
    CUDA_TRY(cudaGetLastError());
    return 0;
}

int check_built(elses_system s) {
    if (!s) return fail(ELSES_ERR_ARG, "null system");
    if (s->n <= 0 || !s->H.p) return fail(ELSES_ERR_STATE, "system not built");
    return 0;
}

ReduceArgs reduce_args(elses_system s) {
    ReduceArgs r{};
    r.M = s->M;
    r.nu_max = s->nu_max;
    r.eps = s->eps.p;
    r.c = s->cc.p;
    r.d = s->dd.p;
    r.g = s->gg.p;
    r.nu_eff = s->nu_eff.p;
    r.kT = s->p.kT;
    r.inv_kT = 1.0 / s->p.kT;
    r.n_electrons = s->p.n_electrons;
    r.tol = s->p.mu_tol;
    r.max_iter = s->p.max_bisect;
    r.state = s->bstate.p;
    r.partials = s->partials.p;
    r.ticket = s->ticket.p;
    r.act = s->act.p;
    r.act_n = s->act_n.p;
    r.act_below = s->act_below.p;
    return r;
}

DensityArgs density_args(elses_system s, double mu, double* rho, double* rhoE) {
    DensityArgs d{};
    d.row_ptr = s->row_ptr.p;
    d.tmap = s->tmap.p;
    d.nu_max = s->nu_max;
    d.eps = s->eps.p;
    d.c = s->cc.p;
    d.nu_eff = s->nu_eff.p;
    d.mu = mu;
    d.kT = s->p.kT;
    d.rho = rho;
    d.rhoE = rhoE;
    return d;
}

// rho columns of atoms [b, e) at mu: from V where it is formed, else from the eigen-factors of the
// batch just computed (t = V w formed by k_eig_weights).
static void density_batch(elses_system s, double mu, double* rho, double* rhoE, int b, int e, const double* V,
                          int v0, const double* UP, int u0, bool factors, cudaStream_t st,
                          const double* mu_dev = nullptr) {
    DensityArgs d = density_args(s, mu, rho, rhoE);
    d.mu_dev = mu_dev;
    d.atom_begin = b;
    d.atom_end = e;
    d.V = V;
    d.v_col0 = v0;
    d.UP = UP;
    d.up_block0 = u0;
    s->tic(T_DENSITY, st);
    if (factors) {
        eig_density_weights(eig_args(s, b, e, nullptr), mu, mu_dev, s->p.kT, s->ewt.p, st);
        s->stats.launches++;
        d.T = s->ewt.p;
    }
    density_columns(d, st);
    s->toc(st);
    s->stats.launches++;
}

// rho columns of every atom at mu from the archive: t = V w of every column in one launch (from
// V for the columns the pool could not hold), then the density.
static void density_archived(elses_system s, double mu, double* rho, double* rhoE, cudaStream_t st,
                             const double* mu_dev) {
    DensityArgs d = density_args(s, mu, rho, rhoE);
    d.mu_dev = mu_dev;
    d.atom_begin = 0;
    d.atom_end = s->n;
    d.V = s->V.p;
    d.v_col0 = 0;
    d.UP = s->UP.p;
    d.up_block0 = 0;
    s->tic(T_DENSITY, st);
    eig_density_weights_archived(eig_args(s, 0, s->n, s->V.p), mu, mu_dev, s->p.kT, s->ewt_all.p, st);
    d.T = s->ewt_all.p;
    density_columns(d, st);
    s->toc(st);
    s->stats.launches += 2;
}

// mu_dev: when set, mu is read from device memory (the captured step of the graph form).
int density_impl(elses_system s, double mu, double* rho, double* rhoE, cudaStream_t st,
                 const double* mu_dev) {
    if (s->atoms_done != s->n) return fail(ELSES_ERR_STATE, "density_matrix needs every column");
    if (!mu_dev) TRY(clear_status(s, st));
    if (!s->p.two_pass && s->v_arch) {
        density_archived(s, mu, rho, rhoE, st, mu_dev);
    } else if (!s->p.two_pass) {
        density_batch(s, mu, rho, rhoE, 0, s->n, s->V.p, 0, s->UP.p, 0, s->v_lazy, st, mu_dev);
    } else {
        // second calculation of G (Eq. 3): recompute every batch, then its rho columns
        for (int b = 0; b < s->n; b += s->batch_atoms) {
            const int e = std::min(s->n, b + s->batch_atoms);
            double* V;
            double* UP;
            int v0, u0;
            TRY(run_batch(s, b, e, false, &V, &v0, &UP, &u0, st, true, false));
            density_batch(s, mu, rho, rhoE, b, e, V, v0, UP, u0, true, st, mu_dev);
        }
    }
    return 0;
}

int energy_force_eager(elses_system s, double* mu_host, double* e_band_host, double* f_free_host,
                       double* forces_dev, cudaStream_t st) {
    void* stream = (void*)st;
    int warn = elses_green_columns(s, 0, s->M, 0, nullptr, nullptr, nullptr, stream);
    if (warn < 0) return warn;
    double mu = 0.0;
    TRY(elses_find_mu(s, &mu, nullptr, stream));
    TRY(density_impl(s, mu, s->rho.p, s->rhoE.p, st));
    s->have_rho = true;
    ReduceArgs r = reduce_args(s);
    s->tic(T_BISECT, st);
    scalars_at(r, mu, st);
    s->toc(st);
    s->stats.launches++;
    if (forces_dev) {
        const double* gh = s->rho.p;
        const double* gs = s->rhoE.p;
        if (s->p.force_mode == 1) {   // exact gradient of the truncated method: dF/dH, -dF/dS
            TRY(s->adjH.ensure((size_t)s->nnzb * 16));
            TRY(s->adjS.ensure((size_t)s->nnzb * 16));
            TRY(adjoint_impl(s, mu, 0, s->n, s->adjH.p, s->adjS.p, -1.0, st));
            gh = s->adjH.p;
            gs = s->adjS.p;
        }
        s->tic(T_FORCE, st);
        forces(s->pos.p, s->n, s->box, s->skd, s->row_ptr.p, s->col_idx.p, s->row_of.p, s->tmap.p, s->nnzb,
               gh, gs, s->gblock.p, forces_dev, st);
        s->toc(st);
        s->stats.launches += 2;
    }
    BisectState h{};
    CUDA_TRY(cudaMemcpyAsync(&h, s->bstate.p, sizeof h, cudaMemcpyDeviceToHost, st));
    int rc = check_status(s, st);
    if (rc < 0) return rc;
    if (mu_host) *mu_host = mu;
    if (e_band_host) *e_band_host = h.e_band;
    if (f_free_host) *f_free_host = h.omega + mu * s->p.n_electrons;
    return warn > 0 ? warn : rc;
}

}  // namespace elses

extern "C" {

int elses_density_matrix(elses_system s, double mu, double* rho_dev, double* rhoE_dev, void* stream) {
    NvtxRange nvtx_range("elses_density_matrix");
    TRY(check_built(s));
    if (!rho_dev) return fail(ELSES_ERR_ARG, "null rho");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(density_impl(s, mu, rho_dev, rhoE_dev, st));
    return check_status(s, st);
}

int elses_energies(elses_system s, double mu, double* n_host, double* e_band_host, double* omega_host,
                   double* f_free_host, void* stream) {
    NvtxRange nvtx_range("elses_energies");
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    if (s->atoms_done != s->n) return fail(ELSES_ERR_STATE, "energies need every column");
    ReduceArgs r = reduce_args(s);
    s->tic(T_BISECT, st);
    scalars_at(r, mu, st);
    s->toc(st);
    s->stats.launches++;
    BisectState h{};
    CUDA_TRY(cudaMemcpyAsync(&h, s->bstate.p, sizeof h, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());   // a failed launch is reported before the timings are read
    s->collect();
    if (n_host) *n_host = h.n_at;
    if (e_band_host) *e_band_host = h.e_band;
    if (omega_host) *omega_host = h.omega;
    if (f_free_host) *f_free_host = h.omega + mu * s->p.n_electrons;
    return ELSES_OK;
}


int elses_version(void) { return 1; }

const char* elses_last_error(void) { return g_err.c_str(); }

void elses_system_destroy(elses_system s) {
    if (!s) return;
    // the device buffers are freed by their destructors
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
        cudaEventDestroy(s->ev_fork);
        cudaEventDestroy(s->ev_join);
    }
    delete s;
}

int elses_build_clusters(elses_system* sys, int n_atoms, const double* pos_dev,
                         const double* box_host, const elses_sk* sk, const elses_params* params,
                         void* stream) {
    NvtxRange nvtx_range("elses_build_clusters");
    cudaStream_t st = (cudaStream_t)stream;
    if (!sys || !pos_dev || !box_host || !sk || !params) return fail(ELSES_ERR_ARG, "null argument");
    if (n_atoms <= 0) return fail(ELSES_ERR_ARG, "n_atoms must be positive");
    elses_params p = *params;
    if (p.breakdown_tol <= 0) p.breakdown_tol = 1e-12;
    if (p.mu_tol <= 0) p.mu_tol = 1e-13;
    if (p.max_bisect <= 0) p.max_bisect = 100;
    if (p.max_neighbors <= 0) p.max_neighbors = 64;
    if (p.max_cluster <= 0) p.max_cluster = 512;
    if (p.nu < 1 || p.nu > kMaxNu) return fail(ELSES_ERR_ARG, "nu must be in [1, %d]", kMaxNu);
    if (p.n_classes < 0 || p.n_classes > 4) return fail(ELSES_ERR_ARG, "n_classes must be in [0, 4]");
    for (int c = 0; c < p.n_classes; ++c)
        if (p.class_nu[c] < 1 || p.class_nu[c] > kMaxNu) return fail(ELSES_ERR_ARG, "class_nu out of range");
    if (!(p.kT > 0)) return fail(ELSES_ERR_ARG, "kT must be positive");
    if (p.force_mode < 0 || p.force_mode > 1) return fail(ELSES_ERR_ARG, "force_mode must be 0 or 1");
    if (p.krylov_block < 0 || p.krylov_block > 1) return fail(ELSES_ERR_ARG, "krylov_block must be 0 or 1");
    if (p.batch_atoms < 0) return fail(ELSES_ERR_ARG, "batch_atoms must be >= 0");
    if (p.k3_lanes != 0 && p.k3_lanes != 32) return fail(ELSES_ERR_ARG, "k3_lanes must be 0 or 32");
    if (p.max_qr_sweeps < 0) return fail(ELSES_ERR_ARG, "max_qr_sweeps must be >= 0");
    if (p.reorth != 0 && p.reorth != 1) return fail(ELSES_ERR_ARG, "reorth must be 0 or 1");
    if (p.keep_factors < 0) return fail(ELSES_ERR_ARG, "keep_factors must be 0 or positive");
    if (p.krylov_block) {
        if (p.nu < 4) return fail(ELSES_ERR_ARG, "a block space needs nu >= 4");
        for (int c = 0; c < p.n_classes; ++c)
            if (p.class_nu[c] < 4) return fail(ELSES_ERR_ARG, "a block space needs nu >= 4");
        if (p.force_mode == 1) return fail(ELSES_ERR_NOT_IMPLEMENTED, "exact forces need per-column spaces");
    }
    if (!(sk->r_cut > sk->r_on) || !(sk->r_on > 0)) return fail(ELSES_ERR_ARG, "need 0 < r_on < r_cut");
    for (int d = 0; d < 3; ++d) {
        if (!(box_host[d] > 2.0 * sk->r_cut)) return fail(ELSES_ERR_ARG, "box must exceed 2*r_cut");
        if (p.r_cluster > 0 && !(box_host[d] > 2.0 * p.r_cluster))
            return fail(ELSES_ERR_ARG, "box must exceed 2*r_cluster");
    }
    if (p.r_cluster > 0 && p.r_cluster < sk->r_cut)
        return fail(ELSES_ERR_ARG, "r_cluster must be >= r_cut (the pattern rows lie in the cluster)");
    elses_system s = *sys;
    if (s && s->n != n_atoms) return fail(ELSES_ERR_ARG, "rebuild with a different atom count");
    if (!s) {
        s = new elses_system_s();
        *sys = s;
    }
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev));
    s->n = n_atoms;
    s->M = 4 * n_atoms;
    std::memcpy(s->box, box_host, sizeof s->box);
    s->sk = *sk;
    s->p = p;
    s->user_hs = false;
    s->skd.Es = sk->Es;
    s->skd.Ep = sk->Ep;
    for (int x = 0; x < 4; ++x) {
        s->skd.V0[x] = sk->V0[x];
        s->skd.qH[x] = sk->qH[x];
        s->skd.S0[x] = sk->S0[x];
        s->skd.qS[x] = sk->qS[x];
    }
    s->skd.r0 = sk->r0;
    s->skd.r_on = sk->r_on;
    s->skd.r_cut = sk->r_cut;
    s->collect();
    s->stats = elses_stats{};
    const int n = n_atoms;
    TRY(s->pos.ensure(3 * (size_t)n));
    CUDA_TRY(cudaMemcpyAsync(s->pos.p, pos_dev, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    TRY(s->counters.ensure(kCounters));
    CUDA_TRY(cudaMemsetAsync(s->counters.p, 0, sizeof(int) * kCounters, st));
    TRY(s->flops_ctr.ensure(2));   // [0] Krylov kernels, [1] exact-gradient kernels
    CUDA_TRY(cudaMemsetAsync(s->flops_ctr.p, 0, 2 * sizeof(unsigned long long), st));
    check_finite(s->pos.p, 3 * n, s->counters.p + 2, st);
    s->stats.launches++;
    {
        int h = 0;
        CUDA_TRY(cudaMemcpyAsync(&h, s->counters.p + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (h) return fail(ELSES_ERR_NONFINITE, "positions contain NaN or Inf");
    }

    // cell grid with edges >= r_cut
    CellGrid& g = s->grid;
    g.ncell = 1;
    for (int d = 0; d < 3; ++d) {
        g.L[d] = box_host[d];
        g.nc[d] = std::max(1, std::min(256, (int)std::floor(box_host[d] / sk->r_cut)));
        g.len[d] = box_host[d] / g.nc[d];
        g.ncell *= g.nc[d];
    }
    TRY(s->cell_of.ensure(n));
    TRY(s->cell_count.ensure(g.ncell));
    TRY(s->cell_start.ensure(g.ncell + 1));
    TRY(s->cursor.ensure(g.ncell));
    TRY(s->cell_atoms.ensure(n));
    build_cells(s->pos.p, n, g, s->cell_of.p, s->cell_count.p, s->cell_start.p, s->cursor.p,
                s->cell_atoms.p, st);
    s->stats.launches += 4;

    // neighbour pattern and clusters: both lists counted (the cluster one beside the neighbour
    // one on the second stream), one readback, then both filled side by side
    TRY(s->row_cnt.ensure(n));
    TRY(s->row_ptr.ensure(n + 1));
    const bool clusters = p.r_cluster > 0;
    if (clusters) {
        TRY(s->cl_cnt.ensure(n));
        TRY(s->cl_ptr.ensure(n + 1));
    }
    count_lists(s->pos.p, n, g, s->cell_of.p, s->cell_start.p, s->cell_atoms.p, sk->r_cut,
                s->row_cnt.p, s->counters.p + 0, st);
    scan_exclusive(s->row_cnt.p, s->row_ptr.p, n, st);
    s->stats.launches += 2;
    if (clusters) {
        TRY(fork_side(s, st));
        count_lists(s->pos.p, n, g, s->cell_of.p, s->cell_start.p, s->cell_atoms.p, p.r_cluster,
                    s->cl_cnt.p, s->counters.p + 1, s->side);
        scan_exclusive(s->cl_cnt.p, s->cl_ptr.p, n, s->side);
        TRY(join_side(s, st));
        s->stats.launches += 2;
    }
    int hc[2] = {0, 0};
    std::vector<int> hp;
    CUDA_TRY(cudaMemcpyAsync(hc, s->counters.p, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    s->h_row_ptr.resize(n + 1);
    CUDA_TRY(cudaMemcpyAsync(s->h_row_ptr.data(), s->row_ptr.p, sizeof(int) * (n + 1),
                             cudaMemcpyDeviceToHost, st));
    if (clusters) {
        hp.resize(n + 1);
        CUDA_TRY(cudaMemcpyAsync(hp.data(), s->cl_ptr.p, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    s->max_nb = hc[0];
    s->nnzb = s->h_row_ptr[n];
    if (s->max_nb > p.max_neighbors)
        return fail(ELSES_ERR_CAPACITY, "an atom has %d neighbours (max_neighbors %d)", s->max_nb, p.max_neighbors);
    TRY(s->col_idx.ensure(s->nnzb));
    TRY(s->row_of.ensure(s->nnzb));
    TRY(s->tmap.ensure(s->nnzb));
    if (clusters) {
        s->max_cl = hc[1];
        s->cl_total = hp[n];
        if (s->max_cl > p.max_cluster)
            return fail(ELSES_ERR_CAPACITY, "a cluster has %d atoms (max_cluster %d)", s->max_cl, p.max_cluster);
        TRY(s->cl_idx.ensure(std::max(1, hp[n])));
        s->h_clsize.resize(n);
        for (int i = 0; i < n; ++i) s->h_clsize[i] = hp[i + 1] - hp[i];
        TRY(fork_side(s, st));
        fill_lists(s->pos.p, n, g, s->cell_of.p, s->cell_start.p, s->cell_atoms.p, p.r_cluster,
                   s->cl_ptr.p, s->cl_idx.p, p.max_cluster, s->counters.p + 2, s->side);
        s->stats.launches++;
    } else {
        if (n > p.max_cluster)
            return fail(ELSES_ERR_CAPACITY, "whole-system cluster of %d atoms exceeds max_cluster %d", n, p.max_cluster);
        s->max_cl = n;
        s->cl_total = (long long)n * n;
        s->h_clsize.assign(n, n);
    }
    fill_lists(s->pos.p, n, g, s->cell_of.p, s->cell_start.p, s->cell_atoms.p, sk->r_cut,
               s->row_ptr.p, s->col_idx.p, p.max_neighbors, s->counters.p + 2, st);
    s->stats.launches++;

    // Slater-Koster H and S
    TRY(s->H.ensure((size_t)s->nnzb * 16));
    TRY(s->S.ensure((size_t)s->nnzb * 16));
    TRY(s->skr.ensure((size_t)s->nnzb * 12));
    sk_build(s->pos.p, n, s->box, s->skd, s->row_ptr.p, s->col_idx.p, s->nnzb, s->row_of.p, s->tmap.p,
             s->H.p, s->S.p, s->skr.p, st);
    s->stats.launches += 2;
    if (clusters) TRY(join_side(s, st));   // the cluster lists
    TRY(check_status(s, st));
    TRY(prepare_columns(s));
    if (s->p.autotune && s->tuned_bps.empty() && s->p.k3_ctas_per_sm <= 0) TRY(autotune_impl(s, st));
    return ELSES_OK;
}

// A caller's block pattern: checked on the host (rows ascending, inside [0, N), the diagonal
// present, symmetric, rows within max_neighbors), then row map and transpose map, and the
// column buffers sized for it.
static int adopt_pattern(elses_system s, int nnzb, const int* row_ptr_dev, const int* col_idx_dev, cudaStream_t st) {
    const int n = s->n;
    std::vector<int> rp(n + 1), ci((size_t)nnzb);
    CUDA_TRY(cudaMemcpyAsync(rp.data(), row_ptr_dev, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(ci.data(), col_idx_dev, sizeof(int) * (size_t)nnzb, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (rp[0] != 0 || rp[n] != nnzb) return fail(ELSES_ERR_ARG, "row_ptr must run from 0 to nnzb");
    int max_row = 0;
    for (int i = 0; i < n; ++i) {
        const int a = rp[i], b = rp[i + 1];
        if (b < a) return fail(ELSES_ERR_ARG, "row_ptr must not decrease (row %d)", i);
        max_row = std::max(max_row, b - a);
        bool diag = false;
        for (int e = a; e < b; ++e) {
            if (ci[e] < 0 || ci[e] >= n) return fail(ELSES_ERR_ARG, "col_idx out of range (row %d)", i);
            if (e > a && ci[e] <= ci[e - 1]) return fail(ELSES_ERR_ARG, "row %d is not strictly ascending", i);
            diag |= ci[e] == i;
        }
        if (!diag) return fail(ELSES_ERR_ARG, "row %d has no diagonal block", i);
    }
    if (max_row > s->p.max_neighbors)
        return fail(ELSES_ERR_CAPACITY, "a row has %d blocks (max_neighbors %d)", max_row, s->p.max_neighbors);
    if (s->p.r_cluster > 0) {   // each column's pattern rows must lie in its cluster
        int* cnt = s->counters.p + 3;
        CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int), st));
        pattern_outside_clusters(n, row_ptr_dev, col_idx_dev, s->cl_ptr.p, s->cl_idx.p, cnt, st);
        s->stats.launches++;
        int outside = 0;
        CUDA_TRY(cudaMemcpyAsync(&outside, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (outside) return fail(ELSES_ERR_ARG, "%d pattern blocks join atoms farther apart than r_cluster", outside);
    }
    std::vector<int> row_of((size_t)nnzb), tmap((size_t)nnzb);
    for (int i = 0; i < n; ++i)
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            row_of[e] = i;
            const int J = ci[e];
            const auto first = ci.begin() + rp[J], last = ci.begin() + rp[J + 1];
            const auto it = std::lower_bound(first, last, i);
            if (it == last || *it != i) return fail(ELSES_ERR_ARG, "the pattern is not symmetric (%d, %d)", i, J);
            tmap[e] = (int)(it - ci.begin());
        }
    TRY(s->col_idx.ensure(nnzb));
    TRY(s->row_of.ensure(nnzb));
    TRY(s->tmap.ensure(nnzb));
    TRY(s->H.ensure((size_t)nnzb * 16));
    TRY(s->S.ensure((size_t)nnzb * 16));
    CUDA_TRY(cudaMemcpyAsync(s->row_ptr.p, rp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(s->col_idx.p, ci.data(), sizeof(int) * (size_t)nnzb, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(s->row_of.p, row_of.data(), sizeof(int) * (size_t)nnzb, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(s->tmap.p, tmap.data(), sizeof(int) * (size_t)nnzb, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors are released on return
    s->h_row_ptr = rp;
    s->nnzb = nnzb;
    s->max_nb = max_row;
    return 0;
}

int elses_set_hs(elses_system s, int nnzb, const int* row_ptr_dev, const int* col_idx_dev, const double* H_dev,
                 const double* S_dev, void* stream) {
    NvtxRange nvtx_range("elses_set_hs");
    TRY(check_built(s));
    if (!H_dev || !S_dev) return fail(ELSES_ERR_ARG, "null H or S");
    if ((row_ptr_dev == nullptr) != (col_idx_dev == nullptr))
        return fail(ELSES_ERR_ARG, "row_ptr and col_idx go together");
    cudaStream_t st = (cudaStream_t)stream;
    if (row_ptr_dev) {
        if (nnzb < s->n) return fail(ELSES_ERR_ARG, "nnzb must cover at least the diagonal blocks");
        TRY(adopt_pattern(s, nnzb, row_ptr_dev, col_idx_dev, st));   // checks before it changes anything
        s->user_hs = true;
        s->drop_graph();
        TRY(prepare_columns(s));
    }
    s->user_hs = true;
    CUDA_TRY(cudaMemcpyAsync(s->H.p, H_dev, sizeof(double) * 16 * s->nnzb, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(s->S.p, S_dev, sizeof(double) * 16 * s->nnzb, cudaMemcpyDeviceToDevice, st));
    s->have_rho = false;
    s->v_lazy = false;   // every column is recomputed before V is used again
    s->v_arch = false;
    s->atom_done.assign(s->n, 0);
    s->atoms_done = 0;
    s->have_mu = false;
    return ELSES_OK;
}

int elses_green_columns(elses_system s, int col_begin, int col_end, int n_z, const double* z_host,
                        double* G_dev, int* nu_eff_dev, void* stream) {
    NvtxRange nvtx_range("elses_green_columns");
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    if (col_begin < 0 || col_end > s->M || col_begin > col_end || col_begin % 4 || col_end % 4)
        return fail(ELSES_ERR_ARG, "column range must be whole atoms inside [0, M)");
    if (n_z < 0 || (n_z > 0 && (!z_host || !G_dev))) return fail(ELSES_ERR_ARG, "bad z / G arguments");
    TRY(clear_status(s, st));
    if (n_z > 0) {
        TRY(s->zbuf.ensure(2 * (size_t)n_z));
        CUDA_TRY(cudaMemcpyAsync(s->zbuf.p, z_host, sizeof(double) * 2 * n_z, cudaMemcpyHostToDevice, st));
    }
    const int a0 = col_begin / 4, a1 = col_end / 4;
    const bool stored = !s->p.two_pass;
    if (stored && s->arch && n_z == 0 && a0 == 0 && a1 == s->n) TRY(reset_archive(s, st));
    // the batches of the launch plan that meet [a0, a1), each from its first atom (the atoms of
    // it before a0 are recomputed as well: the same columns again) to the range's end in it
    for (int b = a0 / s->batch_atoms * s->batch_atoms; b < a1; b += s->batch_atoms) {
        const int e = std::min(a1, b + s->batch_atoms);
        double* V;
        double* UP;
        int v0, u0;
        // first calculation of G in the two-pass workflow keeps only the spectra; V is formed
        // only for G(z) (or, stored, later where something needs it)
        TRY(run_batch(s, b, e, stored, &V, &v0, &UP, &u0, st, stored || n_z > 0, n_z > 0));
        if (n_z > 0) {
            DensityArgs d = density_args(s, 0.0, nullptr, nullptr);
            d.atom_begin = std::max(b, a0);
            d.atom_end = e;
            d.V = V;
            d.v_col0 = v0;
            d.UP = UP;
            d.up_block0 = u0;
            d.n_z = n_z;
            d.z = s->zbuf.p;
            d.G = G_dev;
            green_columns_eval(d, st);
            s->stats.launches++;
        }
        for (int a = b; a < e; ++a)
            if (!s->atom_done[a]) { s->atom_done[a] = 1; s->atoms_done++; }
    }
    if (nu_eff_dev && a1 > a0)
        CUDA_TRY(cudaMemcpyAsync(nu_eff_dev + col_begin, s->nu_eff.p + col_begin,
                                 sizeof(int) * (col_end - col_begin), cudaMemcpyDeviceToDevice, st));
    s->have_mu = false;
    return check_status(s, st);
}

int elses_find_mu(elses_system s, double* mu_host, double* n_at_mu_host, void* stream) {
    NvtxRange nvtx_range("elses_find_mu");
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    if (s->atoms_done != s->n) return fail(ELSES_ERR_STATE, "find_mu needs every column (call green_columns first)");
    ReduceArgs r = reduce_args(s);
    s->tic(T_BISECT, st);
    bisect_init(r, st);
    s->stats.launches += 3;
    for (int it = 0; it < s->p.max_bisect; ++it) bisect_step(r, st);
    s->stats.launches += s->p.max_bisect;
    s->toc(st);
    BisectState h{};
    CUDA_TRY(cudaMemcpyAsync(&h, s->bstate.p, sizeof h, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());
    s->collect();
    s->stats.bisect_steps = h.iter;
    if (h.status & DEV_NONFINITE) return fail(ELSES_ERR_NONFINITE, "non-finite poles");
    if (h.status & DEV_NO_BRACKET)
        return fail(ELSES_ERR_NO_BRACKET, "N(lo)=%.17g N(hi)=%.17g do not bracket N_e=%.17g", h.n_lo, h.n_hi,
                    s->p.n_electrons);
    s->mu = h.mu;
    s->have_mu = true;
    if (mu_host) *mu_host = h.mu;
    if (n_at_mu_host) {
        s->tic(T_BISECT, st);
        scalars_at(r, h.mu, st);
        s->toc(st);
        s->stats.launches++;
        CUDA_TRY(cudaMemcpyAsync(&h, s->bstate.p, sizeof h, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        CUDA_TRY(cudaGetLastError());
        s->collect();
        *n_at_mu_host = h.n_at;
    }
    return ELSES_OK;
}

int elses_energy_force(elses_system s, double* mu_host, double* e_band_host, double* f_free_host,
                       double* forces_dev, void* stream) {
    NvtxRange nvtx_range("elses_energy_force");
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    if (forces_dev && s->user_hs) return fail(ELSES_ERR_STATE, "forces need the Slater-Koster H, S");
    if (s->p.graph) return energy_force_graph(s, mu_host, e_band_host, f_free_host, forces_dev, st);
    return energy_force_eager(s, mu_host, e_band_host, f_free_host, forces_dev, st);
}

int elses_cohp_spectrum(elses_system s, int n_z, const double* z_host, double* C_dev, double* Csig_dev,
                        double* Cpi_dev, double* dos_host, void* stream) {
    NvtxRange nvtx_range("elses_cohp_spectrum");
    TRY(check_built(s));
    if (n_z <= 0 || !z_host) return fail(ELSES_ERR_ARG, "need n_z > 0 energies");
    if (!C_dev && !Csig_dev && !Cpi_dev && !dos_host) return fail(ELSES_ERR_ARG, "no output requested");
    if ((Csig_dev || Cpi_dev) && s->user_hs)
        return fail(ELSES_ERR_STATE, "the sigma / pi split needs the Slater-Koster H");
    if (s->atoms_done != s->n) return fail(ELSES_ERR_STATE, "the spectra need every column");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(clear_status(s, st));
    TRY(s->zbuf.ensure(2 * (size_t)n_z));
    CUDA_TRY(cudaMemcpyAsync(s->zbuf.p, z_host, sizeof(double) * 2 * n_z, cudaMemcpyHostToDevice, st));
    if (dos_host) {
        TRY(s->dosbuf.ensure(dos_scratch_doubles(n_z)));
        dos_at(reduce_args(s), s->zbuf.p, n_z, s->dosbuf.p, st);
        s->stats.launches += 2;
    }
    if (C_dev || Csig_dev || Cpi_dev) {
        // G on the pattern for a chunk of energies at a time (at most 256 MB), then Eq. 4
        const size_t per_z = (size_t)s->nnzb * 16 * 2;
        const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n_z, (size_t(1) << 25) / per_z));
        TRY(s->gbuf.ensure(per_z * chunk));
        if (!s->p.two_pass) TRY(ensure_V(s, st));
        for (int iz0 = 0; iz0 < n_z; iz0 += chunk) {
            const int nzc = std::min(chunk, n_z - iz0);
            for (int b = 0; b < s->n; b += s->batch_atoms) {
                const int e = std::min(s->n, b + s->batch_atoms);
                DensityArgs d = density_args(s, 0.0, nullptr, nullptr);
                d.atom_begin = b;
                d.atom_end = e;
                if (s->p.two_pass) {   // the second calculation of G for this batch
                    double *V = nullptr, *UP = nullptr;
                    int v0 = 0, u0 = 0;
                    TRY(run_batch(s, b, e, false, &V, &v0, &UP, &u0, st));
                    d.V = V;
                    d.v_col0 = v0;
                    d.UP = UP;
                    d.up_block0 = u0;
                } else {
                    d.V = s->V.p;
                    d.v_col0 = 0;
                    d.UP = s->UP.p;
                    d.up_block0 = 0;
                }
                d.n_z = nzc;
                d.z = s->zbuf.p + 2 * (size_t)iz0;
                d.G = s->gbuf.p;
                green_columns_eval(d, st);
                s->stats.launches++;
            }
            cohp_spectrum(s->pos.p, s->box, s->skd, s->col_idx.p, s->row_of.p, s->nnzb, s->H.p, s->gbuf.p, nzc,
                          iz0, n_z, C_dev, Csig_dev, Cpi_dev, st);
            s->stats.launches++;
        }
    }
    int rc = check_status(s, st);
    if (rc < 0) return rc;
    if (dos_host) {
        const double* dos = s->dosbuf.p + dos_scratch_doubles(n_z) - n_z;
        CUDA_TRY(cudaMemcpyAsync(dos_host, dos, sizeof(double) * n_z, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    return rc;
}

int elses_omega_gradient(elses_system s, double mu, int atom_begin, int atom_end, double* dH_dev,
                         double* dS_dev, void* stream) {
    NvtxRange nvtx_range("elses_omega_gradient");
    TRY(check_built(s));
    if (!dH_dev || !dS_dev) return fail(ELSES_ERR_ARG, "null gradient outputs");
    if (atom_begin < 0 || atom_end > s->n || atom_begin > atom_end)
        return fail(ELSES_ERR_ARG, "atom range [%d, %d) outside [0, %d)", atom_begin, atom_end, s->n);
    if (s->p.krylov_block)
        return fail(ELSES_ERR_NOT_IMPLEMENTED, "the exact gradient is built for per-column Krylov spaces");
    if (s->atoms_done != s->n) return fail(ELSES_ERR_STATE, "the gradient needs every column computed");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(clear_status(s, st));
    TRY(adjoint_impl(s, mu, atom_begin, atom_end, dH_dev, dS_dev, 1.0, st));
    const int rc = check_status(s, st);
    s->collect();
    return rc;
}

int elses_forces(elses_system s, double* forces_dev, void* stream) {
    NvtxRange nvtx_range("elses_forces");
    TRY(check_built(s));
    if (!forces_dev) return fail(ELSES_ERR_ARG, "null forces");
    if (s->user_hs) return fail(ELSES_ERR_STATE, "forces need the Slater-Koster H, S");
    if (!s->have_rho) return fail(ELSES_ERR_STATE, "forces need rho from elses_energy_force");
    cudaStream_t st = (cudaStream_t)stream;
    const double* gh = s->rho.p;
    const double* gs = s->rhoE.p;
    if (s->p.force_mode == 1) {
        TRY(s->adjH.ensure((size_t)s->nnzb * 16));
        TRY(s->adjS.ensure((size_t)s->nnzb * 16));
        TRY(adjoint_impl(s, s->mu, 0, s->n, s->adjH.p, s->adjS.p, -1.0, st));
        gh = s->adjH.p;
        gs = s->adjS.p;
    }
    s->tic(T_FORCE, st);
    forces(s->pos.p, s->n, s->box, s->skd, s->row_ptr.p, s->col_idx.p, s->row_of.p, s->tmap.p, s->nnzb,
           gh, gs, s->gblock.p, forces_dev, st);
    s->toc(st);
    s->stats.launches += 2;
    CUDA_TRY(cudaGetLastError());
    return ELSES_OK;
}

int elses_icohp(elses_system s, const double* rho_dev, double* B_dev, double* Bsig_dev, double* Bpi_dev,
                void* stream) {
    NvtxRange nvtx_range("elses_icohp");
    TRY(check_built(s));
    if (!rho_dev || !B_dev) return fail(ELSES_ERR_ARG, "null rho or B");
    if ((Bsig_dev || Bpi_dev) && s->user_hs)
        return fail(ELSES_ERR_STATE, "the sigma / pi split needs the Slater-Koster H");
    icohp(s->pos.p, s->box, s->skd, s->col_idx.p, s->row_of.p, s->nnzb, s->H.p, rho_dev, B_dev, Bsig_dev,
          Bpi_dev, (cudaStream_t)stream);
    s->stats.launches++;
    CUDA_TRY(cudaGetLastError());
    return ELSES_OK;
}

int elses_get_pattern(elses_system s, int* nnzb_host, int* row_ptr_dev, int* col_idx_dev, void* stream) {
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    if (nnzb_host) *nnzb_host = s->nnzb;
    if (row_ptr_dev)
        CUDA_TRY(cudaMemcpyAsync(row_ptr_dev, s->row_ptr.p, sizeof(int) * (s->n + 1), cudaMemcpyDeviceToDevice, st));
    if (col_idx_dev)
        CUDA_TRY(cudaMemcpyAsync(col_idx_dev, s->col_idx.p, sizeof(int) * s->nnzb, cudaMemcpyDeviceToDevice, st));
    return ELSES_OK;
}

int elses_get_hs(elses_system s, double* H_dev, double* S_dev, void* stream) {
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    if (H_dev) CUDA_TRY(cudaMemcpyAsync(H_dev, s->H.p, sizeof(double) * 16 * s->nnzb, cudaMemcpyDeviceToDevice, st));
    if (S_dev) CUDA_TRY(cudaMemcpyAsync(S_dev, s->S.p, sizeof(double) * 16 * s->nnzb, cudaMemcpyDeviceToDevice, st));
    return ELSES_OK;
}

int elses_get_clusters(elses_system s, long long* total_host, int* max_cluster_host, int* cl_ptr_dev,
                       int* cl_idx_dev, void* stream) {
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    if (total_host) *total_host = s->cl_total;
    if (max_cluster_host) *max_cluster_host = s->max_cl;
    if (s->p.r_cluster > 0) {
        if (cl_ptr_dev)
            CUDA_TRY(cudaMemcpyAsync(cl_ptr_dev, s->cl_ptr.p, sizeof(int) * (s->n + 1), cudaMemcpyDeviceToDevice, st));
        if (cl_idx_dev)
            CUDA_TRY(cudaMemcpyAsync(cl_idx_dev, s->cl_idx.p, sizeof(int) * s->cl_total, cudaMemcpyDeviceToDevice, st));
    }
    return ELSES_OK;
}

int elses_get_spectra(elses_system s, int* nu_max_host, double* eps_dev, double* c_dev, double* d_dev,
                      double* g_dev, int* nu_eff_dev, void* stream) {
    TRY(check_built(s));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)s->M * s->nu_max;
    if (nu_max_host) *nu_max_host = s->nu_max;
    if (eps_dev) CUDA_TRY(cudaMemcpyAsync(eps_dev, s->eps.p, bytes, cudaMemcpyDeviceToDevice, st));
    if (c_dev) CUDA_TRY(cudaMemcpyAsync(c_dev, s->cc.p, bytes, cudaMemcpyDeviceToDevice, st));
    if (d_dev) CUDA_TRY(cudaMemcpyAsync(d_dev, s->dd.p, bytes, cudaMemcpyDeviceToDevice, st));
    if (g_dev) CUDA_TRY(cudaMemcpyAsync(g_dev, s->gg.p, bytes, cudaMemcpyDeviceToDevice, st));
    if (nu_eff_dev) CUDA_TRY(cudaMemcpyAsync(nu_eff_dev, s->nu_eff.p, sizeof(int) * s->M, cudaMemcpyDeviceToDevice, st));
    return ELSES_OK;
}

int elses_get_stats(elses_system s, elses_stats* out) {
    if (!s || !out) return fail(ELSES_ERR_ARG, "null argument");
    *out = s->stats;
    out->k3_ctas_per_sm = s->k3_bps;
    if (s->flops_ctr.p) {
        unsigned long long f[2] = {0, 0};
        CUDA_TRY(cudaMemcpy(f, s->flops_ctr.p, sizeof f, cudaMemcpyDeviceToHost));
        out->krylov_flops = (double)f[0];
        out->adjoint_flops = (double)f[1];
    }
    out->batches = s->batch_atoms > 0 ? (s->n + s->batch_atoms - 1) / s->batch_atoms : 0;
    out->kept_rotations = 0;
    out->v_formed_columns = 0;
    if (s->arch) {
        unsigned long long k[2] = {0, 0};
        CUDA_TRY(cudaMemcpy(k, s->acnt.p, sizeof k, cudaMemcpyDeviceToHost));
        out->kept_rotations = (long long)std::min<unsigned long long>(k[0], s->arch_cap);
        out->v_formed_columns = (long long)k[1];
    }
    out->keep_factors = s->arch ? 1 : 0;
    return ELSES_OK;
}

int elses_reset_stats(elses_system s) {
    if (!s) return fail(ELSES_ERR_ARG, "null system");
    s->collect();
    s->stats = elses_stats{};
    if (s->flops_ctr.p) CUDA_TRY(cudaMemset(s->flops_ctr.p, 0, 2 * sizeof(unsigned long long)));
    return ELSES_OK;
}

int elses_probe_fp64(double* gflops_host, void* stream) {
    if (!gflops_host) return fail(ELSES_ERR_ARG, "null output");
    double g = 0.0;
    const int rc = probe_fp64(&g, (cudaStream_t)stream);
    if (rc != 0) return fail(ELSES_ERR_CUDA, "fp64 probe failed: %s", cudaGetErrorString((cudaError_t)rc));
    *gflops_host = g;
    return ELSES_OK;
}

}  // extern "C"
