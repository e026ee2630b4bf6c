// Allocation-free Hutchinson trace of one polynomial (mpmc_trace_poly_noalloc).
//
// Some callers cannot call cudaMalloc: an application whose framework owns
// the whole device through its own caching allocator (so a raw cudaMalloc
// would fail or fragment that pool), or a caller on a latency-critical path
// where cudaMalloc's implicit device synchronisation is not acceptable.  This
// entry point runs the same root-form stencil chain as mpmc_trace_levels for
// a single polynomial, but keeps every intermediate in one file-scope device
// array of fixed size, so it calls no allocating routine at all.
#include "mpmc.h"
#include "kernels.h"

#include <cmath>
#include <complex>
#include <mutex>

using namespace mpmc;

namespace {

// The scratch array.  Every GPU that loads the library holds it until the
// process exits.  In host code `g_scratch` is only a host-side stand-in for
// the symbol, never a device address: its device address is looked up once
// per device with cudaGetSymbolAddress and that pointer is what the kernels get.
static __device__ __align__(256) unsigned char g_scratch[MPMC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
void* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_scratch on the current device (set-up on first use).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return MPMC_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return MPMC_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return MPMC_ECUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return MPMC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
    int nb;
    size_t off_links, off_stage, off_w0, off_w1, off_acc, off_samples, total;
    LaunchCfg cfg;
};

// Carve the scratch for a block of nb columns; total > capacity means "does not fit".
Plan plan_for(const Geom& g, int nb, bool host_links) {
    Plan p;
    p.nb = nb;
    p.cfg = chain_config(g, nb, 64, 1);
    const size_t links = (size_t)g.V * 36 * 16;
    const size_t vec = (size_t)g.V * 12 * nb * 16;
    size_t o = 0;
    p.off_links = o; o = align256(o + links);
    p.off_stage = o; o = align256(o + (host_links ? links : 0));
    p.off_w0 = o; o = align256(o + vec);
    p.off_w1 = o; o = align256(o + vec);
    p.off_acc = o; o = align256(o + (size_t)p.cfg.gx * nb * 16);
    p.off_samples = o; o = align256(o + (size_t)nb * 16);
    p.total = o;
    return p;
}

}  // namespace

extern "C" MPMC_API int mpmc_trace_poly_noalloc(const int dims[4], const double* links, double kappa, int bc_t,
                                                const double* roots, int nroots, uint64_t seed, int level,
                                                int first, int nsamples, double* samples, int on_device,
                                                void* stream_) {
    if (!dims || !links || !roots || !samples) return MPMC_EINVAL;
    for (int d = 0; d < 4; ++d)
        if (dims[d] < 2 || dims[d] > 4096) return MPMC_EINVAL;
    if (!std::isfinite(kappa) || (bc_t != 1 && bc_t != -1)) return MPMC_EINVAL;
    if (nroots < 1 || nroots > 100000 || nsamples < 1 || first < 0 || level < 0) return MPMC_EINVAL;
    for (int i = 0; i < nroots; ++i) {
        const std::complex<double> z(roots[2 * i], roots[2 * i + 1]);
        if (!std::isfinite(z.real()) || !std::isfinite(z.imag()) || z == 0.0) return MPMC_ENONFINITE;
    }
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V * 12 > (1LL << 31) - 1) return MPMC_EINVAL;
    Geom g{dims[0], dims[1], dims[2], dims[3], (int)V, bc_t};
    const bool host = on_device == 0;
    // the widest block (<= 64 columns) whose working set fits the fixed array
    int nb = nsamples < 64 ? nsamples : 64;
    while (nb > 1 && plan_for(g, nb, host).total > (size_t)MPMC_NOALLOC_SCRATCH_BYTES) nb /= 2;
    const Plan p = plan_for(g, nb, host);
    if (p.total > (size_t)MPMC_NOALLOC_SCRATCH_BYTES) return MPMC_EINVAL;   // lattice too large for the array

    void* base = nullptr;
    if (int rc = scratch_address(&base)) return rc;
    unsigned char* S = static_cast<unsigned char*>(base);
    cudaStream_t st = (cudaStream_t)stream_;
    const double n = 12.0 * (double)V;

    // links -> kernel layout in the scratch (host links staged in the scratch first)
    const double* src = links;
    if (host) {
        if (cudaMemcpyAsync(S + p.off_stage, links, (size_t)V * 36 * 16, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return MPMC_ECUDA;
        src = reinterpret_cast<const double*>(S + p.off_stage);
    }
    launch_links(ST_F64, g.V, src, S + p.off_links, st);

    void* w[2] = {S + p.off_w0, S + p.off_w1};
    double2* acc = reinterpret_cast<double2*>(S + p.off_acc);
    double2* smp = reinterpret_cast<double2*>(S + p.off_samples);
    const std::complex<double> th0(roots[0], roots[1]);
    const std::complex<double> cst = n / th0;
    for (int b0 = 0; b0 < nsamples; b0 += nb) {
        const int nvalid = nsamples - b0 < nb ? nsamples - b0 : nb;
        const NoiseSpec ns{seed, (uint32_t)level, (uint32_t)(first + b0)};
        // the array keeps the previous call's contents: accumulators start from zero
        if (cudaMemsetAsync(acc, 0, (size_t)p.cfg.gx * nb * 16, st) != cudaSuccess) return MPMC_ECUDA;
        const void* in = nullptr;   // first step reads the noise itself
        for (int j = 1; j < nroots; ++j) {
            const std::complex<double> al = 1.0 / std::complex<double>(roots[2 * (j - 1)], roots[2 * (j - 1) + 1]);
            const std::complex<double> wnext = 1.0 / std::complex<double>(roots[2 * j], roots[2 * j + 1]);
            StepArgs a{};
            a.in = in;
            a.out = w[(j - 1) % 2];
            a.ymode = 0;
            a.dot = true;
            a.alpha[0] = al.real(); a.alpha[1] = al.imag();
            a.kappa = kappa;
            a.dot_w[0] = wnext.real(); a.dot_w[1] = wnext.imag();
            a.acc = acc;
            launch_step(ST_F64, g, S + p.off_links, nb, ns, a, p.cfg, st);
            in = a.out;
        }
        const double chi[2] = {cst.real(), cst.imag()}, clo[2] = {0.0, 0.0};
        launch_finalize(p.cfg.gx, nb, nvalid, acc, nullptr, chi, clo, nullptr, smp, nullptr, nullptr, st);
        if (cudaGetLastError() != cudaSuccess) return MPMC_ECUDA;
        if (cudaMemcpyAsync(samples + 2 * (size_t)b0, smp, (size_t)nvalid * 16,
                            host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return MPMC_ECUDA;
    }
    if (host && cudaStreamSynchronize(st) != cudaSuccess) return MPMC_ECUDA;
    return MPMC_OK;
}
