// The CUDA-graph form of elses_energy_force (params.graph): the step's device work enqueued
// without host synchronisation, captured once and replayed while its key is unchanged.
#include <cstddef>
#include <cstring>
#include <vector>

#include "system_impl.h"

using namespace elses;

namespace elses {

// The device work of one energy + force evaluation, enqueued with no host synchronisation (the
// captured step of the graph form): the columns, the bisection's fixed sequence of launches
// (those after convergence return at once), the density, the scalars and the forces, all at the
// mu the bisection leaves in device memory. The same kernels and arguments as the eager path.
int enqueue_step(elses_system s, double* forces_dev, cudaStream_t st) {
    TRY(clear_status(s, st));
    const bool stored = !s->p.two_pass;
    if (stored && s->arch) TRY(reset_archive(s, st));
    for (int b = 0; b < s->n; b += s->batch_atoms) {
        const int e = std::min(s->n, b + s->batch_atoms);
        double *V = nullptr, *UP = nullptr;
        int v0 = 0, u0 = 0;
        TRY(run_batch(s, b, e, stored, &V, &v0, &UP, &u0, st, stored, false));
    }
    s->atom_done.assign(s->n, 1);
    s->atoms_done = s->n;
    ReduceArgs r = reduce_args(s);
    s->tic(T_BISECT, st);
    bisect_init(r, st);
    for (int it = 0; it < s->p.max_bisect; ++it) bisect_step(r, st);
    s->toc(st);
    s->stats.launches += 3 + s->p.max_bisect;
    const double* mu_dev = (const double*)((const char*)s->bstate.p + offsetof(BisectState, mu));
    TRY(density_impl(s, 0.0, s->rho.p, s->rhoE.p, st, mu_dev));
    s->tic(T_BISECT, st);
    scalars_at_state(r, st);
    s->toc(st);
    s->stats.launches++;
    if (forces_dev) {
        const double* gh = s->rho.p;
        const double* gs = s->rhoE.p;
        if (s->p.force_mode == 1) {
            TRY(adjoint_impl(s, 0.0, 0, s->n, s->adjH.p, s->adjS.p, -1.0, st, mu_dev));
            gh = s->adjH.p;
            gs = s->adjS.p;
        }
        s->tic(T_FORCE, st);
        forces(s->pos.p, s->n, s->box, s->skd, s->row_ptr.p, s->col_idx.p, s->row_of.p, s->tmap.p, s->nnzb,
               gh, gs, s->gblock.p, forces_dev, st);
        s->toc(st);
        s->stats.launches += 2;
    }
    return 0;
}

// What a captured step depends on besides device data: the buffers (allocation epoch), the
// forces output, the parameters and the Krylov launch plan.
std::vector<long long> graph_key(elses_system s, const double* forces_dev) {
    std::vector<long long> k = {(long long)g_alloc_epoch, (long long)(uintptr_t)forces_dev, s->n, s->nnzb,
                                s->nu_max, s->na_max, s->batch_atoms, s->user_hs ? 1 : 0, s->max_nb,
                                s->max_cl, s->deg_cap};
    auto add_bytes = [&k](const void* src, size_t bytes) {
        std::vector<long long> w((bytes + 7) / 8, 0);
        std::memcpy(w.data(), src, bytes);
        k.insert(k.end(), w.begin(), w.end());
    };
    add_bytes(&s->p, sizeof(elses_params));
    add_bytes(s->box, sizeof(s->box));
    add_bytes(&s->skd, sizeof(s->skd));
    for (int b = 0; b < s->n; b += s->batch_atoms) k.push_back(s->h_row_ptr[b]);   // batch pattern offsets
    for (const auto& L : s->k3_launches) {
        k.insert(k.end(), {L.batch_begin, L.batch_end, L.item_begin, L.item_count, L.na, L.grid, L.bps,
                           (long long)L.scratch_off});
    }
    return k;
}

int capture_step(elses_system s, double* forces_dev) {
    s->drop_graph();
    if (!s->gstream) CUDA_TRY(cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
    if (!s->side) {   // the second stream and its events exist before the capture
        TRY(fork_side(s, s->gstream));
        TRY(join_side(s, s->gstream));
        CUDA_TRY(cudaStreamSynchronize(s->gstream));
    }
    const long long l0 = s->stats.launches, c0 = s->stats.columns, k0 = s->stats.krylov_launches;
    CUDA_TRY(cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeRelaxed));
    s->capturing = true;
    int rc = enqueue_step(s, forces_dev, s->gstream);
    s->capturing = false;
    s->graph_v_lazy = s->v_lazy;
    s->graph_v_arch = s->v_arch;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s->gstream, &g);
    s->graph_launches = s->stats.launches - l0;
    s->graph_krylov = s->stats.krylov_launches - k0;
    s->graph_columns = s->stats.columns - c0;
    s->stats.launches = l0;            // counted at every replay
    s->stats.columns = c0;
    s->stats.krylov_launches = k0;
    if (rc >= 0 && ce != cudaSuccess) rc = fail(ELSES_ERR_CUDA, "stream capture: %s", cudaGetErrorString(ce));
    if (rc >= 0 && cudaGraphInstantiate(&s->graph_exec, g, 0) != cudaSuccess) {
        s->graph_exec = nullptr;
        rc = fail(ELSES_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (g) cudaGraphDestroy(g);
    if (rc < 0) s->drop_graph();
    return rc;
}

// The graph form: the first call with a new plan runs the eager path (and checks it), the next
// captures the step, later calls replay it; one host synchronisation per call.
int energy_force_graph(elses_system s, double* mu_host, double* e_band_host, double* f_free_host,
                       double* forces_dev, cudaStream_t st) {
    if (!s->graph_exec || graph_key(s, forces_dev) != s->graph_key) {
        if (graph_key(s, forces_dev) != s->graph_key) {
            s->drop_graph();
            const int rc = energy_force_eager(s, mu_host, e_band_host, f_free_host, forces_dev, st);
            if (rc >= 0) s->graph_key = graph_key(s, forces_dev);
            return rc;
        }
        CUDA_TRY(cudaStreamSynchronize(st));   // the capture only records; nothing runs
        TRY(capture_step(s, forces_dev));
    }
    CUDA_TRY(cudaGraphLaunch(s->graph_exec, st));
    s->stats.launches += s->graph_launches;
    s->stats.krylov_launches += s->graph_krylov;
    s->stats.columns += s->graph_columns;
    // the host-side state the captured step leaves (a rebuild since the capture reset it): every
    // column computed, V formed or left to the kept factors as at the capture
    s->atom_done.assign(s->n, 1);
    s->atoms_done = s->n;
    s->v_lazy = s->graph_v_lazy;
    s->v_arch = s->graph_v_arch;
    s->have_rho = true;
    BisectState h{};
    CUDA_TRY(cudaMemcpyAsync(&h, s->bstate.p, sizeof h, cudaMemcpyDeviceToHost, st));
    const int rc = check_status(s, st);
    s->collect_graph();
    s->stats.bisect_steps = h.iter;
    if (h.status & DEV_NONFINITE) return fail(ELSES_ERR_NONFINITE, "non-finite poles");
    if (h.status & DEV_NO_BRACKET)
        return fail(ELSES_ERR_NO_BRACKET, "N(lo)=%.17g N(hi)=%.17g do not bracket N_e=%.17g", h.n_lo, h.n_hi,
                    s->p.n_electrons);
    if (rc < 0) return rc;
    s->mu = h.mu;
    s->have_mu = true;
    if (mu_host) *mu_host = h.mu;
    if (e_band_host) *e_band_host = h.e_band;
    if (f_free_host) *f_free_host = h.omega + h.mu * s->p.n_electrons;
    return rc;
}

}  // namespace elses
