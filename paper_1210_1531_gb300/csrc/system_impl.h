// Private header of the host runtime (system.cu, autotune.cu, graph.cu): the system handle's
// state, its device buffers and the helpers the runtime files share.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"


namespace elses {
// Records the message of the last error (elses_last_error) and returns code.
int fail(int code, const char* fmt, ...);

// An NVTX range over one library call, named after the call (shown by Nsight Systems and other
// NVTX tools; header-only NVTX 3, a no-op when no tool is attached). Closed on every return.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace elses

#define CUDA_TRY(x)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) return elses::fail(ELSES_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

#define TRY(x)                     \
    do {                           \
        int r_ = (x);              \
        if (r_ < 0) return r_;     \
    } while (0)

// Bumped by every device (re)allocation of a DevBuf: a captured graph whose buffers may have
// moved is captured again.
extern unsigned long long g_alloc_epoch;

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;
    int ensure(size_t n) {
        if (n <= cap && p) return 0;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(n, 1);
        if (cudaMalloc(&p, want * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return elses::fail(ELSES_ERR_OOM, "device allocation of %zu bytes failed", want * sizeof(T));
        }
        cap = want;
        ++g_alloc_epoch;
        return 0;
    }
    void release() {   // a captured graph that used the buffer is then out of date
        if (p) {
            cudaFree(p);
            ++g_alloc_epoch;
        }
        p = nullptr;
        cap = 0;
    }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
};

struct elses_system_s {
    int n = 0, M = 0;
    double box[3] = {0, 0, 0};
    elses_sk sk{};
    elses_params p{};
    elses::SKDev skd{};
    int num_sms = 0;
    elses::CellGrid grid{};
    bool user_hs = false;

    DevBuf<double> pos;
    DevBuf<int> cell_of, cell_count, cell_start, cursor, cell_atoms;
    DevBuf<int> row_cnt, row_ptr, col_idx, row_of, tmap;
    DevBuf<int> cl_cnt, cl_ptr, cl_idx;
    DevBuf<int> counters;   // see kCounters
    DevBuf<unsigned long long> flops_ctr;
    DevBuf<double> H, S, skr;
    int nnzb = 0, max_nb = 0, max_cl = 0;
    long long cl_total = 0;
    std::vector<int> h_row_ptr;

    int nu_max = 0, na_max = 0, k3_grid = 0, batch_atoms = 0, deg_cap = 0, k3_bps = 0;
    std::vector<int> tuned_bps;            // autotuner: resident Krylov CTAs per SM by class capacity / 16
    std::vector<int> tuned_order;          // autotuner: work-queue order by class capacity / 16 (1 size, 2 atom)
    std::vector<int> tuned_half;           // autotuner: odd 16-slot classes, 1 half-warps, 2 whole warps
    // Krylov launches: per batch of atoms, one launch per cluster size class (slots of 32 atoms),
    // each with its own shared-memory footprint and resident-CTA count
    // scratch_off: where the launch's per-CTA scratch starts, so that the class launches of one
    // batch can run at the same time
    // key: the class's bound on cluster size in slots of 16 atoms (its capacity na may be larger)
    struct K3Launch { int batch_begin, batch_end, item_begin, item_count, na, grid, bps, half, key; size_t scratch_off; };
    cudaStream_t side = nullptr;           // second stream for concurrent class launches
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<K3Launch> k3_launches;
    std::vector<int> h_clsize;
    DevBuf<double> kscratch, Hp, Sp, urow, surow, hurow, etri, efac, erot_c, erot_s, ewt;
    DevBuf<unsigned char> erot_k;
    DevBuf<int> erot_n, eperm;
    DevBuf<double> eps, cc, dd, gg, V, UP, Vb, UPb;
    DevBuf<int> nu_eff, order;
    DevBuf<double> rho, rhoE, gblock;
    DevBuf<double> ascratch, adjH, adjS;   // exact-gradient scratch and its pattern gradients
    DevBuf<unsigned long long> adj_acc;    // their exact fixed-point sums (AdjointArgs::acc)
    DevBuf<double> bstore;                 // per-column bases kept for the exact gradient
    size_t bstride = 0, bvec = 0;
    bool use_store = false;
    // the eigen-factors of every column are in the batch buffers and the stored V is not formed
    bool v_lazy = false;
    // several batches: their eigen-factors kept in an archive of every column (EigArgs::ar) in
    // place of V formed per batch; arch: the archive is planned, v_arch: the stored V of the
    // archived columns is not formed (columns the pool could not hold have V)
    DevBuf<double> afac, arot_c, arot_s, ewt_all;
    DevBuf<unsigned char> arot_k;
    DevBuf<int> aperm, an, alist;
    DevBuf<unsigned long long> aoff, acnt;
    unsigned long long arch_cap = 0;
    size_t arch_M = 0;
    int arch_nm = 0;
    bool arch = false, v_arch = false, arch_init = false;
    std::vector<int> adj_bps;              // resident adjoint CTAs per SM, by cluster slots
    DevBuf<double> partials, zbuf, gbuf, dosbuf, act_below;
    DevBuf<double2> act;
    DevBuf<int> act_n;
    DevBuf<elses::BisectState> bstate;
    DevBuf<unsigned> ticket;
    std::vector<char> atom_done;
    long long atoms_done = 0;

    elses_stats stats{};
    double mu = 0.0;
    bool have_mu = false;
    bool have_rho = false;   // rho, rhoE of the current positions are in rho / rhoE

    // CUDA-event timing of kernel groups (params.timing = 1)
    struct EvPair { cudaEvent_t a, b; int cat; };
    std::vector<EvPair> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t ev() {
        cudaEvent_t e;
        if (!pool.empty()) { e = pool.back(); pool.pop_back(); }
        else cudaEventCreate(&e);
        return e;
    }
    // while a step is captured into the graph form, the timing events become event-record
    // nodes of the graph (recorded at every replay, read by collect_graph)
    bool capturing = false;
    std::vector<EvPair> graph_ev;
    void tic(int cat, cudaStream_t st) {
        if (!p.timing) return;
        EvPair q{ev(), ev(), cat};
        if (capturing) {
            cudaEventRecordWithFlags(q.a, st, cudaEventRecordExternal);
            graph_ev.push_back(q);
        } else {
            cudaEventRecord(q.a, st);
            pending.push_back(q);
        }
    }
    void toc(cudaStream_t st) {
        if (!p.timing) return;
        if (capturing) {
            if (!graph_ev.empty()) cudaEventRecordWithFlags(graph_ev.back().b, st, cudaEventRecordExternal);
            return;
        }
        if (pending.empty()) return;
        cudaEventRecord(pending.back().b, st);
    }
    void add_time(const EvPair& q) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
            double* slot[] = {&stats.t_krylov_ms, &stats.t_eig_ms, &stats.t_bisect_ms,
                              &stats.t_density_ms, &stats.t_force_ms, &stats.t_adjoint_ms};
            *slot[q.cat] += ms;
        }
    }
    void collect_graph() {   // after a synchronisation of the stream that replayed the graph
        for (auto& q : graph_ev) add_time(q);
        cudaGetLastError();
    }
    // graph form of elses_energy_force (params.graph): the captured step, what it was captured
    // for (launch plan, buffers, forces output, parameters), the kernels it launches
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t gstream = nullptr;       // capture stream (the legacy stream cannot capture)
    std::vector<long long> graph_key;
    long long graph_launches = 0, graph_krylov = 0, graph_columns = 0;
    bool graph_v_lazy = false;            // v_lazy as the captured step leaves it
    bool graph_v_arch = false;            // and v_arch
    void drop_graph() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        graph_exec = nullptr;
        for (auto& q : graph_ev) { pool.push_back(q.a); pool.push_back(q.b); }
        graph_ev.clear();
    }
    // after a synchronisation of the stream and a check of cudaGetLastError (it clears the error
    // that an unrecorded timing event leaves)
    void collect() {
        for (auto& q : pending) {
            add_time(q);
            pool.push_back(q.a);
            pool.push_back(q.b);
        }
        pending.clear();
        cudaGetLastError();
    }
    ~elses_system_s() {
        drop_graph();
        if (gstream) cudaStreamDestroy(gstream);
        for (auto& q : pending) { pool.push_back(q.a); pool.push_back(q.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

enum { T_KRYLOV = 0, T_EIG = 1, T_BISECT = 2, T_DENSITY = 3, T_FORCE = 4, T_ADJOINT = 5 };
// device counters: [0] max neighbours, [1] max cluster, [2] status, [3] a caller pattern's blocks
// outside the clusters (elses_set_hs), [8..] the work
// queues of the class launches of a batch (one each, so that they can run at the same time)
constexpr int kQueue0 = 8;
constexpr int kCounters = 24;

namespace elses {

// Runtime helpers shared by system.cu, autotune.cu and graph.cu.
int nu_of_params(const elses_params& p);
int check_status(elses_system s, cudaStream_t st, bool allow_breakdown_warning = true);
int clear_status(elses_system s, cudaStream_t st);
int prepare_columns(elses_system s);
int fork_side(elses_system s, cudaStream_t st);
int join_side(elses_system s, cudaStream_t st);
KrylovArgs krylov_args(elses_system s, int b, int e);
EigArgs eig_args(elses_system s, int b, int e, double* V);
int ensure_V(elses_system s, cudaStream_t st);
int reset_archive(elses_system s, cudaStream_t st);
int run_batch(elses_system s, int b, int e, bool stored, double** V_out, int* v_col0,
              double** UP_out, int* up_block0, cudaStream_t st, bool need_rows = true, bool form_v = true);
int adjoint_impl(elses_system s, double mu, int lo, int hi, double* gH, double* gS, double s_scale,
                 cudaStream_t st, const double* mu_dev = nullptr);
int autotune_impl(elses_system s, cudaStream_t st);
int check_built(elses_system s);
ReduceArgs reduce_args(elses_system s);
DensityArgs density_args(elses_system s, double mu, double* rho, double* rhoE);
int density_impl(elses_system s, double mu, double* rho, double* rhoE, cudaStream_t st,
                 const double* mu_dev = nullptr);
int energy_force_eager(elses_system s, double* mu_host, double* e_band_host, double* f_free_host,
                       double* forces_dev, cudaStream_t st);
int energy_force_graph(elses_system s, double* mu_host, double* e_band_host, double* f_free_host,
                       double* forces_dev, cudaStream_t st);

}  // namespace elses
