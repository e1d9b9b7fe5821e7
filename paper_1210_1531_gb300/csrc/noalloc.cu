// Allocation-free chemical-potential bisection (elses_find_mu_static).
//
// The same bisection kernels as elses_find_mu (k_bracket / k_count in reduce.cu) run on
// caller-owned spectra; their scratch -- the per-block partial sums, the bracket state and the
// last-block ticket -- lives in one file-scope static device array instead of device memory
// allocated at run time. The array is part of the library image: every GPU that loads the
// library holds it until the process exits.
//
// Its address is looked up (cudaGetSymbolAddress with the device current) at the start of every
// call, not cached: after cudaDeviceReset the next context loads the module again and the array
// may move, and a cached address would then point at freed memory. The lookup allocates nothing;
// on the first call on a device it may load the library's device code, so that first call should
// come before any stream capture. Every call shares the one array: calls whose work overlaps on
// the GPU (different streams, or several host threads) race on it and must be serialised by the
// caller.
#include "internal.h"

namespace elses {
namespace {

constexpr int kStaticMaxBlocks = 4096;                          // reduction blocks supported
constexpr size_t kStatePart = 4 * (size_t)kStaticMaxBlocks;      // partials: [block][4]
constexpr size_t kStateSlot = 24;                               // bracket state, in doubles
constexpr size_t kStaticDoubles = kStatePart + 32;              // + bracket state + ticket
static_assert(sizeof(BisectState) <= kStateSlot * sizeof(double), "bracket state outgrew its slot");
static_assert(kStateSlot + 1 <= kStaticDoubles - kStatePart, "no room for the ticket");

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

// Device address of the static scratch on the current device (the device must be current).
cudaError_t static_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace elses

using namespace elses;

extern "C" int elses_find_mu_static(int n_columns, int nu_max, const double* eps_dev,
                                    const double* c_dev, const double* d_dev, const double* g_dev,
                                    const int* nu_eff_dev, double kT, double n_electrons,
                                    double mu_tol, int max_bisect, double* mu_host,
                                    double* n_at_mu_host, double* e_band_host, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (n_columns <= 0 || nu_max < 1 || nu_max > kMaxNu)
        return report_error(ELSES_ERR_ARG, "n_columns must be positive and nu_max in [1, %d]", kMaxNu);
    if (!eps_dev || !c_dev || !d_dev || !nu_eff_dev || !mu_host)
        return report_error(ELSES_ERR_ARG, "null spectra or output pointer");
    if (e_band_host && !g_dev) return report_error(ELSES_ERR_ARG, "e_band needs g");
    if (!(kT > 0)) return report_error(ELSES_ERR_ARG, "kT must be positive");
    const int grid = reduce_grid();
    if (grid > kStaticMaxBlocks)
        return report_error(ELSES_ERR_CAPACITY,
                            "this device needs %d reduction blocks; the static scratch holds %d",
                            grid, kStaticMaxBlocks);
    double* base = nullptr;
    cudaError_t e = static_scratch(&base);
    if (e != cudaSuccess)
        return report_error(ELSES_ERR_CUDA, "static scratch lookup failed: %s", cudaGetErrorString(e));
    ReduceArgs r{};
    r.M = n_columns;
    r.nu_max = nu_max;
    r.eps = eps_dev;
    r.c = c_dev;
    r.d = d_dev;
    r.g = g_dev ? g_dev : d_dev;
    r.nu_eff = nu_eff_dev;
    r.kT = kT;
    r.inv_kT = 1.0 / kT;
    r.n_electrons = n_electrons;
    r.tol = mu_tol > 0 ? mu_tol : 1e-13;
    r.max_iter = max_bisect > 0 ? max_bisect : 100;
    r.partials = base;
    r.state = reinterpret_cast<BisectState*>(base + kStatePart);
    r.ticket = reinterpret_cast<unsigned*>(base + kStatePart + kStateSlot);
    // the ticket must start at zero; the state is written by the bracket kernel
    e = cudaMemsetAsync(r.ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return report_error(ELSES_ERR_CUDA, "%s", cudaGetErrorString(e));
    bisect_init(r, st);
    for (int it = 0; it < r.max_iter; ++it) bisect_step(r, st);
    BisectState h{};
    e = cudaMemcpyAsync(&h, r.state, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(ELSES_ERR_CUDA, "%s", cudaGetErrorString(e));
    if (h.status & DEV_NONFINITE) return report_error(ELSES_ERR_NONFINITE, "non-finite poles");
    if (h.status & DEV_NO_BRACKET)
        return report_error(ELSES_ERR_NO_BRACKET, "N(lo)=%.17g N(hi)=%.17g do not bracket N_e=%.17g",
                            h.n_lo, h.n_hi, n_electrons);
    *mu_host = h.mu;
    if (n_at_mu_host || e_band_host) {
        scalars_at(r, h.mu, st);
        e = cudaMemcpyAsync(&h, r.state, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return report_error(ELSES_ERR_CUDA, "%s", cudaGetErrorString(e));
        if (n_at_mu_host) *n_at_mu_host = h.n_at;
        if (e_band_host) *e_band_host = h.e_band;
    }
    return ELSES_OK;
}
