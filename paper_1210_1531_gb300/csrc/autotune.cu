// The autotuner of the Krylov kernel's launch shape (elses_autotune; params.autotune at build).
#include <algorithm>
#include <vector>

#include "system_impl.h"

using namespace elses;

namespace elses {

// The autotuner: per size class (at the first batch that has it), the Krylov kernel timed at every resident
// CTA count that fits, on the class's first atoms in launch order (up to two full waves at the
// largest count); the fastest per atom is kept in tuned_bps. A class of an odd number of 16-atom
// slots is timed in both column forms, half-warp (capacity 16 ns) and whole-warp (16 (ns + 1)),
// whatever the occupancy heuristic would have planned, and the faster kept in tuned_half. With
// the work queue, the whole class is then timed in both orders of its atoms -- decreasing
// cluster size (short tail) and atom order (neighbouring clusters in flight together share H
// and S in L2) -- and the faster is kept in tuned_order. The launches are planned again.
int autotune_impl(elses_system s, cudaStream_t st) {
    const int nm = s->nu_max;
    const int kdeg = s->user_hs ? s->max_nb : s->deg_cap;
    s->tuned_bps.assign(s->na_max / 16 + 1, 0);
    s->tuned_order.assign(s->na_max / 16 + 1, 0);
    s->tuned_half.assign(s->na_max / 16 + 1, 0);
    const bool half_ok = s->p.k3_lanes != 32 && s->p.force_mode == 0 && !s->p.krylov_block;
    // odd classes (an odd number of 16-atom slots) that the occupancy heuristic merged into the
    // next even class are planned on their own for the comparison below, so that half-warp and
    // whole-warp columns are timed for every odd class that has atoms
    if (half_ok) {
        bool split = false;
        for (int a = 0; a < s->n; ++a) {
            const int k = (s->h_clsize[a] + 15) / 16;
            if ((k & 1) && k < (int)s->tuned_half.size() && !s->tuned_half[k]) {
                s->tuned_half[k] = 1;
                split = true;
            }
        }
        if (split) TRY(prepare_columns(s));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    int rc = 0;
    const auto launches = s->k3_launches;
    std::vector<char> seen(s->na_max / 16 + 1, 0);
    for (const auto& L : launches) {
        if (rc || seen[L.key]) continue;   // each class once, at its first batch
        seen[L.key] = 1;
        const int ns = L.key;
        // the kernel forms to compare: a class of an odd number of 16-atom slots runs either
        // with half-warps (capacity 16 ns) or with whole warps (capacity 16 (ns + 1))
        struct Form { int half, na, maxb; };
        std::vector<Form> forms;
        if (half_ok && (ns & 1)) forms = {{1, 16 * ns, 0}, {0, 16 * (ns + 1), 0}};
        else forms = {{L.half, L.na, 0}};
        int maxb_all = 0;
        for (auto& f : forms) {
            f.maxb = s->p.krylov_block ? block_krylov_blocks_per_sm(f.na, kdeg)
                     : f.half          ? krylov_half_blocks_per_sm(f.na, kdeg)
                                       : krylov_blocks_per_sm_max(f.na, kdeg);
            maxb_all = std::max(maxb_all, f.maxb);
            const size_t per_cta = s->p.krylov_block ? block_krylov_scratch_doubles(nm, f.na)
                                                     : (size_t)kWarpsPerAtom * 2 * nm * f.na * 4;
            if ((rc = s->kscratch.ensure((size_t)s->num_sms * f.maxb * per_cta)) < 0) break;
        }
        if (rc) break;
        const int sample = std::min(L.item_count, 2 * s->num_sms * maxb_all);   // the same atoms for every form
        double best = 0.0;
        int best_b = 1, best_f = 0;
        bool first = true;
        for (size_t fi = 0; fi < forms.size() && !rc; ++fi) {
          const Form F = forms[fi];
          for (int b = 1; b <= F.maxb && !rc; ++b) {
            KrylovArgs ka = krylov_args(s, L.batch_begin, L.batch_end);
            ka.UP = nullptr;
            ka.flops = nullptr;
            ka.na_max = F.na;
            ka.half = F.half;
            ka.order = s->order.p + L.item_begin;
            ka.n_items = sample;
            ka.scratch = s->kscratch.p;
            const int grid = std::min(sample, s->num_sms * b);
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {       // the first launch warms caches and clocks
                if (s->p.schedule == 1) {
                    ka.queue = s->counters.p + kQueue0;
                    if (cudaMemsetAsync(ka.queue, 0, sizeof(int), st) != cudaSuccess) { rc = fail(ELSES_ERR_CUDA, "memset"); break; }
                }
                cudaEventRecord(e0, st);
                if (s->p.krylov_block) block_krylov_columns(ka, grid, st);
                else krylov_columns(ka, grid, b, st);
                cudaEventRecord(e1, st);
                s->stats.launches++;
            }
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = fail(ELSES_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            const double per_atom = ms / sample;
            if (first || per_atom < best) { best = per_atom; best_b = b; best_f = (int)fi; first = false; }
          }
        }
        if (!rc && forms.size() == 2) s->tuned_half[ns] = forms[best_f].half ? 1 : 2;
        const int chosen_na = forms[best_f].na, chosen_half = forms[best_f].half;
        if (!rc) s->tuned_bps[ns] = best_b;
        if (rc || s->p.schedule != 1 || L.item_count < 4 * s->num_sms * best_b) continue;
        // queue order of the whole class: as planned (decreasing cluster size), then atom order
        std::vector<int> seg(L.item_count);
        if (cudaMemcpy(seg.data(), s->order.p + L.item_begin, sizeof(int) * L.item_count,
                       cudaMemcpyDeviceToHost) != cudaSuccess) { rc = fail(ELSES_ERR_CUDA, "order readback"); break; }
        std::vector<int> atom_order = seg;
        std::sort(atom_order.begin(), atom_order.end());
        float t_order[2] = {0.f, 0.f};
        for (int o = 0; o < 2 && !rc; ++o) {
            const std::vector<int>& ord = o == 0 ? seg : atom_order;
            if (cudaMemcpyAsync(s->order.p + L.item_begin, ord.data(), sizeof(int) * L.item_count,
                                cudaMemcpyHostToDevice, st) != cudaSuccess) { rc = fail(ELSES_ERR_CUDA, "order upload"); break; }
            KrylovArgs ka = krylov_args(s, L.batch_begin, L.batch_end);
            ka.UP = nullptr;
            ka.flops = nullptr;
            ka.na_max = chosen_na;
            ka.half = chosen_half;
            ka.order = s->order.p + L.item_begin;
            ka.n_items = L.item_count;
            ka.scratch = s->kscratch.p;
            ka.queue = s->counters.p + kQueue0;
            const int grid = std::min(L.item_count, s->num_sms * best_b);
            for (int rep = 0; rep < 2; ++rep) {
                cudaMemsetAsync(ka.queue, 0, sizeof(int), st);
                cudaEventRecord(e0, st);
                if (s->p.krylov_block) block_krylov_columns(ka, grid, st);
                else krylov_columns(ka, grid, best_b, st);
                cudaEventRecord(e1, st);
                s->stats.launches++;
            }
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t_order[o], e0, e1) != cudaSuccess)
                rc = fail(ELSES_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(cudaGetLastError()));
        }
        if (!rc) s->tuned_order[ns] = t_order[1] < t_order[0] ? 2 : 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        s->tuned_bps.clear();
        s->tuned_order.clear();
        s->tuned_half.clear();
        return rc;
    }
    TRY(clear_status(s, st));        // the sampled columns may have flagged a breakdown
    CUDA_TRY(cudaStreamSynchronize(st));
    return prepare_columns(s);       // launch plan with the chosen shapes; columns invalidated
}

}  // namespace elses

extern "C" {

int elses_autotune(elses_system s, int run, int max_classes, int* classes_out, int* n_host, void* stream) {
    NvtxRange nvtx_range("elses_autotune");
    TRY(check_built(s));
    if (max_classes < 0 || (max_classes > 0 && !classes_out)) return fail(ELSES_ERR_ARG, "bad class output");
    if (run) {
        if (s->p.k3_ctas_per_sm > 0) return fail(ELSES_ERR_STATE, "k3_ctas_per_sm fixes the launch shape");
        TRY(autotune_impl(s, (cudaStream_t)stream));
    }
    int n = 0;
    std::vector<char> seen(s->na_max / 16 + 1, 0);
    for (const auto& L : s->k3_launches) {   // every class once, largest first within a batch
        if (seen[L.key]) continue;
        seen[L.key] = 1;
        if (n < max_classes) {
            const int key = L.key;
            const bool by_atom = key < (int)s->tuned_order.size() && s->tuned_order[key] == 2;
            classes_out[3 * n] = L.na;
            classes_out[3 * n + 1] = L.bps;
            classes_out[3 * n + 2] = s->p.schedule != 1 ? 0 : by_atom ? 2 : 1;
        }
        ++n;
    }
    if (n_host) *n_host = n;
    return ELSES_OK;
}

}  // extern "C"
