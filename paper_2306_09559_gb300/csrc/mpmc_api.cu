// Host runtime of the C ABI declared in include/mpmc.h: handle lifetime,
// polynomial chains (root form, composite, projected composite), the level
// engine of the multilevel Monte Carlo and the FP64 Arnoldi setup.
#include "mpmc.h"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using cd = std::complex<double>;
using namespace mpmc;

namespace {

struct PolyDef {
    bool set = false;
    int kind = MPMC_SINGLE;
    std::vector<cd> roots, outer;   // theta (single / inner), eta (outer)
};

// Device work buffers for one storage format and block width.
struct Workspace {
    int storage = -1;
    int nb = 0;
    int V = 0;
    void* w[4] = {nullptr, nullptr, nullptr, nullptr};
    void* y = nullptr;
    void* r = nullptr;        // imported input block / start vectors
    void* x = nullptr;        // output block of apply_poly
    double2* acc_hi = nullptr;
    double2* acc_lo = nullptr;
    int acc_rows = 0;
    size_t acc_cap = 0;       // accumulator entries allocated per buffer
    LaunchCfg cfg{};
    bool sweep = false;       // steps with a memory input use the k_sweep kernels
    SweepCfg sw{};
    bool fast = false;        // ymode-0 steps and outer steps use the issue-lean kernels
    int fast_gx = 0;          // their CTA count along the sites
    bool fsweep = false;      // ... in their t-sweep form (steps with a memory input)
    SweepCfg fsw{};
    uint32_t* words = nullptr;        // Z4 words of the current noise block
    NoiseSpec words_ns{0, 0, 0};
    bool words_ok = false;
};

// TMA tensor map of one input buffer of the t-sweep kernels
struct SweepMap {
    const void* p = nullptr;
    int storage = -1, nb = 0, V = 0, kind = 0;   // kind 0: k_sweep boxes, 1: k_fsweep boxes
    alignas(64) unsigned char m[128];
};

size_t storage_bytes(int st) { return st == ST_F64 ? 16 : (st == ST_F32 ? 8 : 4); }

}  // namespace

struct mpmc_ctx {
    Geom g{};
    double kappa = 0;
    int prec = MPMC_FP64;
    int storage = ST_F64;
    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    void* links64 = nullptr;      // [site][mu][3][3] complex double
    void* links32 = nullptr;      // same in float (FP32 / BF16S handles)
    float4* links_ex = nullptr;   // float links expanded to (re, re, im, im) for the issue-lean kernels
    PolyDef polys[MPMC_MAX_POLYS];
    // deflation
    int k = 0;
    void* Z = nullptr;            // k vectors in the math precision (double or float)
    int* d_pair = nullptr;
    std::vector<cd> lam;
    std::vector<int> pair;
    std::vector<cd> dnorm;        // d_i = z_pair(i)^H gamma5 z_i of the stored vectors
    double2* d_dnorm = nullptr;
    double2* d_coef = nullptr;    // [MPMC_MAX_POLYS][k] c_i / d_i per level
    void* AZ = nullptr;           // A z_i, math precision (projected composite)
    double2* d_Hinv = nullptr;    // (U^H A Z)^{-1}, k x k row-major
    double2* defl_part = nullptr;
    double2* G1 = nullptr;
    double2* G2 = nullptr;
    double2* dterm = nullptr;
    double2* D = nullptr;         // projection coefficients k x nb
    float2* D32 = nullptr;        // the same in FP32
    double2* xz = nullptr;        // b^H Z D per column
    // projected composite (Sec. 4.3): Z and A Z in block layout, H^{-1}, 1/d_i
    void* Zb = nullptr;
    void* Wb = nullptr;
    double2* d_invd = nullptr;
    double2* gram_part = nullptr;
    size_t gram_part_cap = 0;
    bool proj_ready = false;
    int defl_nb = 0;
    // tensor-core deflation dots (reduced-precision handles)
    void* planes = nullptr;       // BF16 hi / lo planes of the deflation vectors, [2][Mpad][Kpad]
    alignas(64) unsigned char tmap[128];
    bool tc_ready = false;
    int use_tc = 1;
    float* tc_part = nullptr;
    size_t tc_part_cap = 0;
    int* d_err = nullptr;         // device flag set by kernels whose bounded waits expired
    // t-sweep stencil: option, t-segment length (0 automatic), tensor maps of input buffers
    // Stencil step classes: bit 0 dotted steps (single / projected chains, incl. the noise-started
    // first step), bit 1 undotted steps (inner steps of composite chains), bit 2 outer steps.
    int use_sweep = 55;           // bits 0-2: t-sweep form of the issue-lean kernels per class; bit 3: k_sweep;
                                  // bit 4: that form with each plane's links staged in shared memory;
                                  // bit 5: its warp-per-site form (blocks of 32 or more columns);
                                  // bit 6: its two-sites-per-warp form
    int sweep_ts = 0;
    int use_fast = 7;             // issue-lean kernels per class (FP32 / BF16S, block widths 16 .. 1024)
    int fast_sl = 1;              // sites per thread of the issue-lean kernels
    long long wait_limit = 4000000000LL;   // bound of each t-sweep mbarrier wait (SM clock cycles, ~2 s)
    int skip_copy = 0;            // failure-detection test hook: t-sweep plane copy left out (0: none)
    int sweep_order = 1;          // launch order of the t-sweep site blocks: 0 plain, 1 Morton curve
    int* blk_order = nullptr;     // device table of that order (made with the first t-sweep shape)
    std::vector<SweepMap> maps;
    // work
    int nb_user = 0;
    int tune_R = 1, tune_bx = 64, tune_sl = 1;   // launch shape of the stencil kernels
    Workspace ws, ws64;
    double2* samples = nullptr;
    size_t samples_cap = 0;
    double* io = nullptr;         // complex-double staging for host I/O
    size_t io_cap = 0;
    double2* kr_part = nullptr;   // Krylov scratch
    double2* kr_h = nullptr;
    double* kr_nrm = nullptr;
    int kr_m = 0;
    long long launches = 0;
    // stochastic rounding of BF16 chain stores: salt of the current chain (from its noise block and
    // polynomial) and the position of the next step in it, so that a call's random bits depend on
    // what it computes, not on the handle's history
    uint32_t sr_base = 0, sr_step = 0;
    double2* probe = nullptr;     // probing: [nchunk][nb] partial sums + 1 total
    size_t probe_cap = 0;
    int* probe_tab = nullptr;     // probing: site colours of the caller's colouring
    size_t probe_tab_cap = 0;
    double2* sol = nullptr;       // solver: basis (m+1 vectors) and 4 work vectors + coefficients
    size_t sol_cap = 0;
    unsigned long long gen = 0;   // bumped by every call that changes what a trace launches
    // profiling: events around kernel launches of each class (mpmc_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::vector<int> ev_cls;
    std::vector<int> ev_var;      // kernel of a stencil launch (PROF_K_*), -1 for other classes
    std::vector<double> ev_bytes;
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long prof_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double prof_b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::string err;
};

namespace {

int fail(mpmc_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_check(mpmc_ctx* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MPMC_OK;
    return fail(h, e == cudaErrorMemoryAllocation ? MPMC_ENOMEM : MPMC_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        int rc__ = cuda_check(h, (call), #call);              \
        if (rc__) return rc__;                                \
    } while (0)

#define LAUNCHED(n)                                                    \
    do {                                                               \
        h->launches += (n);                                            \
        int rc__ = cuda_check(h, cudaGetLastError(), "kernel launch"); \
        if (rc__) return rc__;                                         \
    } while (0)

// Every device buffer of a handle comes from here.  A new allocation bumps the
// handle's generation: a captured batch graph holds the addresses of the
// buffers it was recorded with, and a buffer freed and allocated again (by any
// call on the handle between two batch calls) must force a recapture.
template <class P> int dev_alloc(mpmc_ctx* h, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(h, MPMC_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
    }
    *p = reinterpret_cast<P*>(q);
    if (h) ++h->gen;
    return MPMC_OK;
}

template <class P> void dev_free(P*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

bool finite(cd z) { return std::isfinite(z.real()) && std::isfinite(z.imag()); }

int nsites12(const mpmc_ctx* h) { return 12 * h->g.V; }

void free_ws(Workspace& w) {
    for (auto& p : w.w) dev_free(p);
    dev_free(w.y);
    dev_free(w.r);
    dev_free(w.x);
    dev_free(w.acc_hi);
    dev_free(w.acc_lo);
    dev_free(w.words);
    w.words_ok = false;
    w.acc_cap = 0;
    w.nb = 0;
    w.storage = -1;
}

// Launch shape for the workspace's block; grows the accumulators if needed.
int set_cfg(mpmc_ctx* h, Workspace& w) {
    w.cfg = chain_config(h->g, w.nb, h->tune_bx, h->tune_sl, h->tune_R);
    w.fast = (h->use_fast & 7) && fast_supported(w.storage, w.nb);
    if (w.fast) {
        const int per = fast_sites_per_cta(w.nb) * h->fast_sl;
        w.fast_gx = (h->g.V + per - 1) / per;
    }
    w.fsweep = w.fast && (h->use_sweep & h->use_fast & 7) && fsweep_supported(w.storage, h->g, w.nb);
    if (w.fsweep) w.fsw = fsweep_config(h->g, w.nb, h->sweep_ts, fsweep_variant(h->use_sweep, w.nb));
    if (w.fsweep && !h->blk_order) {
        std::vector<int> order((size_t)w.fsw.nblk);
        fsweep_morton_order(h->g, order.data());
        if (int rc = dev_alloc(h, &h->blk_order, sizeof(int) * order.size())) return rc;
        CK(cudaMemcpy(h->blk_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    }
    w.sweep = (h->use_sweep & 8) && sweep_supported(w.storage, h->g, w.nb);
    if (w.sweep) w.sw = sweep_config(h->g, w.nb, h->sweep_ts);
    // one accumulator row per site block (k_step) or per site block and t-segment (sweep)
    w.acc_rows = std::max(std::max(w.cfg.gx, w.sweep ? w.sw.rows : 0),
                          std::max(w.fast ? w.fast_gx : 0, w.fsweep ? w.fsw.rows : 0));
    const size_t need = (size_t)w.acc_rows * w.nb;
    if (need > w.acc_cap) {
        dev_free(w.acc_hi);
        dev_free(w.acc_lo);
        w.acc_cap = 0;
        if (int rc = dev_alloc(h, &w.acc_hi, sizeof(double2) * need)) return rc;
        if (int rc = dev_alloc(h, &w.acc_lo, sizeof(double2) * need)) return rc;
        w.acc_cap = need;
    }
    return MPMC_OK;
}

int ensure_ws(mpmc_ctx* h, Workspace& w, int storage, int nb) {
    if (w.storage == storage && w.nb == nb) return set_cfg(h, w);
    free_ws(w);
    w.acc_cap = 0;
    const size_t vb = (size_t)h->g.V * 12 * nb * storage_bytes(storage);
    for (auto& p : w.w)
        if (int rc = dev_alloc(h, &p, vb)) return rc;
    if (int rc = dev_alloc(h, &w.y, vb)) return rc;
    if (int rc = dev_alloc(h, &w.r, vb)) return rc;
    if (int rc = dev_alloc(h, &w.x, vb)) return rc;
    if (int rc = dev_alloc(h, &w.words, sizeof(uint32_t) * (size_t)h->g.V * nb)) return rc;
    w.words_ok = false;
    // padding columns must hold finite values: clear everything once
    for (auto& p : w.w) CK(cudaMemsetAsync(p, 0, vb, h->stream));
    CK(cudaMemsetAsync(w.y, 0, vb, h->stream));
    CK(cudaMemsetAsync(w.r, 0, vb, h->stream));
    CK(cudaMemsetAsync(w.x, 0, vb, h->stream));
    w.storage = storage;
    w.nb = nb;
    w.V = h->g.V;
    return set_cfg(h, w);
}

const void* links_for(const mpmc_ctx* h, int storage) { return storage == ST_F64 ? h->links64 : h->links32; }

// kappa as the stencil kernels of a storage format take it.  The reduced-precision links
// are stored premultiplied by kappa (kappa U, formed in FP64 and rounded once per element),
// so those kernels apply A = I - (kappa H) with kappa = 1: a rounded kappa would shift the
// matrix by the same relative amount at every site, a systematic change of every trace,
// while per-element rounding of kappa U varies in sign from element to element.
double kap(const mpmc_ctx* h, int storage) { return storage == ST_F64 ? h->kappa : 1.0; }


// ------------------------------------------------------------------ profiling
int prof_begin(mpmc_ctx* h, int cls, double bytes) {
    if (!h->prof) return MPMC_OK;
    while (h->ev.size() < h->ev_used + 2) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->ev.push_back(e);
    }
    CK(cudaEventRecord(h->ev[h->ev_used], h->stream));
    h->ev_cls.push_back(cls);
    h->ev_var.push_back(-1);
    h->ev_bytes.push_back(bytes);
    return MPMC_OK;
}

int prof_end(mpmc_ctx* h) {
    if (!h->prof) return MPMC_OK;
    CK(cudaEventRecord(h->ev[h->ev_used + 1], h->stream));
    h->ev_used += 2;
    return MPMC_OK;
}

// call after the stream has been synchronised
int prof_collect(mpmc_ctx* h) {
    for (size_t i = 0; i < h->ev_cls.size(); ++i) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]));
        for (int c : {h->ev_cls[i], h->ev_var[i]}) {
            if (c < 0) continue;
            h->prof_ms[c] += ms;
            h->prof_n[c] += 1;
            h->prof_b[c] += h->ev_bytes[i];
        }
    }
    h->ev_cls.clear();
    h->ev_var.clear();
    h->ev_bytes.clear();
    h->ev_used = 0;
    return MPMC_OK;
}

enum { PROF_STENCIL = 0, PROF_DEFLATION = 1, PROF_OTHER = 2 };
// stencil launches by kernel: t-sweep issue-lean, issue-lean, site-parallel, t-sweep site-parallel
enum { PROF_K_FSWEEP = 3, PROF_K_FAST = 4, PROF_K_SITE = 5, PROF_K_SWEEP = 6 };
void prof_variant(mpmc_ctx* h, int var) {
    if (h->prof && !h->ev_var.empty()) h->ev_var.back() = var;
}

double link_bytes(const mpmc_ctx* h, int st) { return (double)h->g.V * 36 * (st == ST_F64 ? 16 : 8); }

// After a synchronisation: ETIMEOUT (and the flag cleared) if a kernel's
// bounded wait on a TMA or tensor-core pipeline gave up.
int device_flag(mpmc_ctx* h) {
    int flag = 0;
    CK(cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(h->d_err, 0, sizeof(int)));
        return fail(h, MPMC_ETIMEOUT, "a bounded device wait gave up (TMA / tensor-core pipeline)");
    }
    return MPMC_OK;
}

// Tensor map of a step input for the t-sweep kernels (made once per buffer, block shape and box).
const void* sweep_map(mpmc_ctx* h, const Workspace& ws, const void* in, int kind) {
    for (const SweepMap& m : h->maps)
        if (m.p == in && m.storage == ws.storage && m.nb == ws.nb && m.V == h->g.V && m.kind == kind) return m.m;
    SweepMap m;
    const bool made = kind ? fsweep_make_map(m.m, ws.storage, in, h->g.V, ws.nb, kind == 2 ? 16 : std::min(ws.nb, 32))
                           : sweep_make_map(m.m, ws.storage, in, h->g.V, ws.nb);
    if (!made) return nullptr;
    m.p = in;
    m.storage = ws.storage;
    m.nb = ws.nb;
    m.V = h->g.V;
    m.kind = kind;
    if (h->maps.size() >= 64) h->maps.erase(h->maps.begin());
    h->maps.push_back(m);
    return h->maps.back().m;
}

uint32_t mix32(uint32_t x) {   // integer mixing for the stochastic-rounding salts
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// Start of a chain: its salt from the noise block (or none, in apply mode) and the polynomial.
void begin_chain(mpmc_ctx* h, const NoiseSpec& ns, uint32_t poly_tag) {
    h->sr_base = mix32((uint32_t)ns.seed ^ mix32((uint32_t)(ns.seed >> 32) ^ mix32(ns.level ^ mix32(ns.j0 ^
                                                                                mix32(poly_tag)))));
    h->sr_step = 0;
}
uint32_t next_salt(mpmc_ctx* h) { return mix32(h->sr_base + 0x9E3779B9u * (h->sr_step++)); }

// Z4 word table of the noise block `ns` for the issue-lean kernels (made when the block changes).
int ensure_words(mpmc_ctx* h, Workspace& ws, const NoiseSpec& ns) {
    if (ws.words_ok && ws.words_ns.seed == ns.seed && ws.words_ns.level == ns.level && ws.words_ns.j0 == ns.j0)
        return MPMC_OK;
    launch_noise_words(h->g, ws.nb, ns, ws.words, h->stream);
    LAUNCHED(1);
    ws.words_ns = ns;
    ws.words_ok = true;
    return MPMC_OK;
}

FastArgs fast_args(const mpmc_ctx* h, const Workspace& ws, double kappa) {
    FastArgs f{};
    fast_geometry(h->g, f);
    f.Ue = h->links_ex;
    f.words = ws.words;
    f.sl = h->fast_sl;
    f.wait_limit = h->wait_limit;
    f.blk_order = h->sweep_order ? h->blk_order : nullptr;
    f.skip_copy = h->skip_copy;
    f.kappa = (float)kappa;
    return f;
}

// One stencil step on the workspace's launch shape: the issue-lean kernels
// (t-sweep form when the input is a stored block and the shape allows it)
// for ymode-0 steps of FP32 / BF16S blocks of the compiled widths, else the
// site-parallel k_step (or k_sweep when selected).
int step_launch(mpmc_ctx* h, Workspace& ws, const StepArgs& a, const NoiseSpec& ns) {
    const int cls = a.dot ? 1 : 2;   // class bit of the step
    if (ws.fast && (h->use_fast & cls) && a.ymode == 0 && !a.op_only && (a.in || a.dot)) {
        const int kind = a.in ? (a.dot ? 1 : 0) : 2;
        if (kind) if (int rc = ensure_words(h, ws, ns)) return rc;
        FastArgs f = fast_args(h, ws, a.kappa);
        f.salt = a.salt;
        f.in = a.in;
        f.out = a.out;
        f.acc = a.acc;
        f.dot_w[0] = a.dot_w[0];
        f.dot_w[1] = a.dot_w[1];
        f.alpha[0] = (float)a.alpha[0];
        f.alpha[1] = (float)a.alpha[1];
        const int var = fsweep_variant(h->use_sweep, ws.nb);
        const void* fmap = (ws.fsweep && (h->use_sweep & cls) && kind < 2) ? sweep_map(h, ws, a.in, var == 1 || var == 3 ? 2 : 1)
                                                                            : nullptr;
        prof_variant(h, fmap ? PROF_K_FSWEEP : PROF_K_FAST);
        if (fmap) {
            if (launch_fsweep(ws.storage, ws.nb, kind, f, ws.fsw, fmap, h->d_err, h->stream, var))
                return fail(h, MPMC_ECUDA, "issue-lean t-sweep step launch failed");
        } else if (launch_fast(ws.storage, ws.nb, kind, f, ws.fast_gx, h->stream)) {
            return fail(h, MPMC_ECUDA, "issue-lean step launch failed");
        }
        return MPMC_OK;
    }
    const void* map = (ws.sweep && a.in) ? sweep_map(h, ws, a.in, 0) : nullptr;
    prof_variant(h, map ? PROF_K_SWEEP : PROF_K_SITE);
    if (map) {
        if (launch_sweep_step(ws.storage, h->g, links_for(h, ws.storage), ws.nb, ns, a, ws.sw, map, h->d_err,
                              h->stream))
            return fail(h, MPMC_ECUDA, "t-sweep step launch failed");
    } else {
        launch_step(ws.storage, h->g, links_for(h, ws.storage), ws.nb, ns, a, ws.cfg, h->stream);
    }
    return MPMC_OK;
}

int do_step(mpmc_ctx* h, Workspace& ws, const StepArgs& a0, const NoiseSpec& ns) {
    StepArgs a = a0;
    a.salt = next_salt(h);
    const int reads = (a.in ? 1 : 0) + (a.ymode == 2 ? 1 : 0);
    const int writes = 1 + (a.ymode ? 1 : 0);
    const double bytes = (double)h->g.V * ws.nb * 12 * storage_bytes(ws.storage) * (reads + writes) + link_bytes(h, ws.storage);
    if (int rc = prof_begin(h, PROF_STENCIL, bytes)) return rc;
    if (int rc = step_launch(h, ws, a, ns)) return rc;
    if (int rc = prof_end(h)) return rc;
    LAUNCHED(1);
    return MPMC_OK;
}

// One outer step (composite chains) on the workspace's launch shape.
int outer_launch(mpmc_ctx* h, Workspace& ws, const OuterArgs& o, const NoiseSpec& ns) {
    if (ws.fast && (h->use_fast & 4)) {
        if (o.dot) if (int rc = ensure_words(h, ws, ns)) return rc;
        FastArgs f = fast_args(h, ws, o.kappa);
        f.salt = o.salt;
        f.in = o.in;
        f.w = o.w;
        f.out = o.wout;
        f.y = o.y;
        f.acc = o.acc;
        f.dot_w[0] = o.dot_w[0];
        f.dot_w[1] = o.dot_w[1];
        for (int i = 0; i < 2; ++i) {
            f.alpha[i] = (float)o.alpha[i];
            f.beta[i] = (float)o.beta[i];
            f.gamma[i] = (float)o.gamma[i];
        }
        const int var = fsweep_variant(h->use_sweep, ws.nb);
        const void* fmap = (ws.fsweep && (h->use_sweep & 4)) ? sweep_map(h, ws, o.in, var == 1 || var == 3 ? 2 : 1) : nullptr;
        prof_variant(h, fmap ? PROF_K_FSWEEP : PROF_K_FAST);
        if (fmap) {
            if (launch_fsweep(ws.storage, ws.nb, o.dot ? 4 : 3, f, ws.fsw, fmap, h->d_err, h->stream, var))
                return fail(h, MPMC_ECUDA, "issue-lean t-sweep outer launch failed");
        } else if (launch_fast(ws.storage, ws.nb, o.dot ? 4 : 3, f, ws.fast_gx, h->stream)) {
            return fail(h, MPMC_ECUDA, "issue-lean outer launch failed");
        }
        return MPMC_OK;
    }
    const void* map = ws.sweep ? sweep_map(h, ws, o.in, 0) : nullptr;
    prof_variant(h, map ? PROF_K_SWEEP : PROF_K_SITE);
    if (map) {
        if (launch_sweep_outer(ws.storage, h->g, links_for(h, ws.storage), ws.nb, ns, o, ws.sw, map, h->d_err,
                               h->stream))
            return fail(h, MPMC_ECUDA, "t-sweep outer launch failed");
    } else {
        launch_outer(ws.storage, h->g, links_for(h, ws.storage), ws.nb, ns, o, ws.cfg, h->stream);
    }
    return MPMC_OK;
}

int do_outer(mpmc_ctx* h, Workspace& ws, const OuterArgs& o0, const NoiseSpec& ns) {
    OuterArgs o = o0;
    o.salt = next_salt(h);
    const double bytes = (double)h->g.V * ws.nb * 12 * storage_bytes(ws.storage) * 5 + link_bytes(h, ws.storage);
    if (int rc = prof_begin(h, PROF_STENCIL, bytes)) return rc;
    if (int rc = outer_launch(h, ws, o, ns)) return rc;
    if (int rc = prof_end(h)) return rc;
    LAUNCHED(1);
    return MPMC_OK;
}

// ------------------------------------------------------------------ roots
std::vector<int> leja_order(const std::vector<cd>& r) {
    const int m = (int)r.size();
    std::vector<int> order;
    if (m == 0) return order;
    std::vector<char> taken(m, 0);
    std::vector<double> score(m, 0.0);
    int first = 0;
    for (int i = 1; i < m; ++i)
        if (std::abs(r[i]) > std::abs(r[first])) first = i;
    order.push_back(first);
    taken[first] = 1;
    for (int step = 1; step < m; ++step) {
        const cd last = r[order.back()];
        int best = -1;
        double bs = -INFINITY;
        for (int i = 0; i < m; ++i) {
            if (taken[i]) continue;
            const double d = std::abs(r[i] - last);
            score[i] += (d > 0) ? std::log(d) : -INFINITY;
            if (best < 0 || score[i] > bs) { best = i; bs = score[i]; }
        }
        order.push_back(best);
        taken[best] = 1;
    }
    return order;
}

// p(lambda) in root form: sum_i theta_i^{-1} prod_{j<i} (1 - lambda/theta_j)
cd poly_value(const std::vector<cd>& th, cd lam) {
    cd w = 1.0, y = 0.0;
    for (size_t i = 0; i < th.size(); ++i) {
        y += w / th[i];
        w *= (1.0 - lam / th[i]);
    }
    return y;
}

cd spec_value(const PolyDef& p, cd lam) {
    if (p.kind == MPMC_SINGLE) return poly_value(p.roots, lam);
    if (p.kind == MPMC_COMPOSITE) {
        const cd pin = poly_value(p.roots, lam);
        return pin * poly_value(p.outer, lam * pin);
    }
    return 1.0 / lam;   // projected composite maps z_i to z_i / lambda_i
}

long long spec_matvecs(const PolyDef& p) {
    const long long m = (long long)p.roots.size();
    if (p.kind == MPMC_SINGLE) return std::max(0LL, m - 1);
    const long long mo = (long long)p.outer.size();
    return (mo - 1) * m + (m - 1);
}

int num_levels(const mpmc_ctx* h) {
    int L = 0;
    while (L < MPMC_MAX_POLYS && h->polys[L].set) ++L;
    return L;
}

inline void setc(double (&d)[2], cd z) { d[0] = z.real(); d[1] = z.imag(); }

// A coefficient as the kernels of a storage format apply it: reduced-precision
// kernels use the FP32 value, so the host uses the same value wherever it
// weights their results (dot weights, closed-form terms).  The chain then
// applies exactly (up to arithmetic rounding) the polynomial with roots
// 1/rnd(1/theta); a correction term below half an FP32 ulp of the result would be
// lost in its rounding, so the coefficients are not split further.  Roots given
// with MPMC_POLY_FP32_COEFS have rnd(1/theta) = 1/theta on every handle, and
// kappa reaches these kernels through links premultiplied by kappa (kappa = 1 in
// the kernels), so that no coefficient is rounded for one precision only.
inline cd rnd(int storage, cd z) {
    if (storage == ST_F64) return z;
    return cd((double)(float)z.real(), (double)(float)z.imag());
}

// ------------------------------------------------------------------ chains
// Trace mode: acc += sum of weighted b^H w over all steps of p(A) applied to
// the start block (noise when start == nullptr); *cst receives the weighted
// b^H w_0 term known in closed form (b^H b = 12 V for noise starts).
int chain_trace(mpmc_ctx* h, Workspace& ws, const PolyDef& p, const NoiseSpec& ns, const void* start,
                double2* acc, cd* cst) {
    begin_chain(h, ns, (uint32_t)(&p - h->polys));
    const int st = ws.storage, nb = ws.nb;
    const void* U = links_for(h, st);
    const double n = (double)nsites12(h);
    const LaunchCfg& cfg = ws.cfg;
    CK(cudaMemsetAsync(acc, 0, sizeof(double2) * (size_t)ws.acc_rows * nb, h->stream));
    *cst = 0.0;
    auto single_from = [&](const std::vector<cd>& th, const void* in0, bool in_is_noise_start) -> int {
        // steps j = 1..m-1 produce w_j with dot weight 1/theta_{j+1}
        const int m = (int)th.size();
        const void* in = in0;
        for (int j = 1; j < m; ++j) {
            StepArgs a{};
            a.in = (j == 1 && in_is_noise_start) ? nullptr : in;
            a.out = ws.w[(j - 1) % 2];
            a.y = nullptr;
            a.ymode = 0;
            a.dot = true;
            const cd al = 1.0 / th[j - 1];
            setc(a.alpha, rnd(st, al));
            a.kappa = kap(h, st);
            setc(a.dot_w, rnd(st, 1.0 / th[j]));
            a.acc = acc;
            if (int rc = do_step(h, ws, a, ns)) return rc;
            in = a.out;
        }
        return MPMC_OK;
    };
    if (p.kind == MPMC_SINGLE) {
        if (start == nullptr) *cst = n * rnd(st, 1.0 / p.roots[0]);
        else return fail(h, MPMC_EINVAL, "internal: single chain from a buffer in trace mode");
        return single_from(p.roots, nullptr, true);
    }
    // composite: outer root form on B = A p_in(A) = I - pi_in(A), then p_in(A) y
    const std::vector<cd>& th = p.roots;
    const std::vector<cd>& eta = p.outer;
    const int m_in = (int)th.size(), m_out = (int)eta.size();
    const size_t ncplx = (size_t)h->g.V * 12 * nb;
    void* Wcur;
    void* Wnxt;
    if (start == nullptr) {
        double one[2] = {1.0, 0.0};
        launch_fill_noise(st, h->g, nb, ns, one, ws.w[2], h->stream);
        LAUNCHED(1);
        Wcur = ws.w[2];
    } else {
        Wcur = const_cast<void*>(start);
    }
    Wnxt = ws.w[3];
    {
        double s1[2];
        setc(s1, rnd(st, 1.0 / eta[0]));
        launch_scale(st, ncplx, Wcur, s1, ws.y, h->stream, next_salt(h));
        LAUNCHED(1);
    }
    if (m_out == 1) {
        // y = b / eta_1; the final chain's first dot is in closed form only for noise starts
        if (start == nullptr) *cst = n * rnd(st, 1.0 / eta[0]) * rnd(st, 1.0 / th[0]);
        else return fail(h, MPMC_ENOTSUP, "internal: projected composite needs at least two outer roots");
    }
    for (int k = 1; k < m_out; ++k) {
        const void* in = Wcur;
        for (int j = 1; j < m_in; ++j) {
            StepArgs a{};
            a.in = in;
            a.out = ws.w[(j - 1) % 2];
            a.ymode = 0;
            a.dot = false;
            const cd al = 1.0 / th[j - 1];
            setc(a.alpha, rnd(st, al));
            a.kappa = kap(h, st);
            if (int rc = do_step(h, ws, a, ns)) return rc;
            in = a.out;
        }
        OuterArgs o{};
        o.in = in;
        o.w = Wcur;
        o.wout = Wnxt;
        o.y = ws.y;
        const cd al = 1.0 / th[m_in - 1];
        setc(o.alpha, rnd(st, al));
        o.kappa = kap(h, st);
        setc(o.beta, rnd(st, 1.0 / eta[k - 1]));
        setc(o.gamma, rnd(st, 1.0 / eta[k]));
        o.dot = (k == m_out - 1);
        setc(o.dot_w, rnd(st, 1.0 / th[0]));
        o.acc = acc;
        if (int rc = do_outer(h, ws, o, ns)) return rc;
        // never write into the caller's start buffer: alternate between w[2] and w[3]
        Wcur = Wnxt;
        Wnxt = (Wcur == ws.w[3]) ? ws.w[2] : ws.w[3];
    }
    // final chain x = p_in(A) y with dots; steps j = 1..m_in-1
    const void* in = ws.y;
    for (int j = 1; j < m_in; ++j) {
        StepArgs a{};
        a.in = in;
        a.out = ws.w[(j - 1) % 2];
        a.ymode = 0;
        a.dot = true;
        const cd al = 1.0 / th[j - 1];
        setc(a.alpha, rnd(st, al));
        a.kappa = kap(h, st);
        setc(a.dot_w, rnd(st, 1.0 / th[j]));
        a.acc = acc;
        if (int rc = do_step(h, ws, a, ns)) return rc;
        in = a.out;
    }
    return MPMC_OK;
}

// Apply mode: X = p(A) B for the block in `in` (storage of ws); X must not alias ws buffers.
int chain_apply_single(mpmc_ctx* h, Workspace& ws, const std::vector<cd>& th, const void* in0, void* X) {
    const int st = ws.storage, nb = ws.nb;
    const void* U = links_for(h, st);
    const NoiseSpec ns{0, 0, 0};
    const int m = (int)th.size();
    const size_t ncplx = (size_t)h->g.V * 12 * nb;
    if (m == 1) {
        double s1[2];
        setc(s1, rnd(st, 1.0 / th[0]));
        launch_scale(st, ncplx, in0, s1, X, h->stream, next_salt(h));
        LAUNCHED(1);
        return MPMC_OK;
    }
    const void* in = in0;
    for (int j = 1; j < m; ++j) {
        StepArgs a{};
        a.in = in;
        a.out = ws.w[(j - 1) % 2];
        a.y = X;
        a.ymode = (j == 1) ? 1 : 2;
        a.dot = false;
        const cd al = 1.0 / th[j - 1];
        setc(a.alpha, rnd(st, al));
        a.kappa = kap(h, st);
        setc(a.ya, rnd(st, 1.0 / th[0]));
        setc(a.yb, rnd(st, 1.0 / th[j]));
        if (int rc = do_step(h, ws, a, ns)) return rc;
        in = a.out;
    }
    return MPMC_OK;
}

int chain_apply(mpmc_ctx* h, Workspace& ws, const PolyDef& p, const void* in0, void* X) {
    begin_chain(h, NoiseSpec{0, 0xA991u, 0}, (uint32_t)(&p - h->polys));
    if (p.kind == MPMC_SINGLE) return chain_apply_single(h, ws, p.roots, in0, X);
    const int st = ws.storage, nb = ws.nb;
    const void* U = links_for(h, st);
    const NoiseSpec ns{0, 0, 0};
    const std::vector<cd>& th = p.roots;
    const std::vector<cd>& eta = p.outer;
    const int m_in = (int)th.size(), m_out = (int)eta.size();
    const size_t ncplx = (size_t)h->g.V * 12 * nb;
    double s1[2];
    setc(s1, rnd(st, 1.0 / eta[0]));
    launch_scale(st, ncplx, in0, s1, ws.y, h->stream, next_salt(h));
    LAUNCHED(1);
    const void* Wcur = in0;
    void* Wnxt = ws.w[2];
    for (int k = 1; k < m_out; ++k) {
        const void* in = Wcur;
        for (int j = 1; j < m_in; ++j) {
            StepArgs a{};
            a.in = in;
            a.out = ws.w[(j - 1) % 2];
            const cd al = 1.0 / th[j - 1];
            setc(a.alpha, rnd(st, al));
            a.kappa = kap(h, st);
            if (int rc = do_step(h, ws, a, ns)) return rc;
            in = a.out;
        }
        OuterArgs o{};
        o.in = in;
        o.w = Wcur;
        o.wout = Wnxt;
        o.y = ws.y;
        const cd al = 1.0 / th[m_in - 1];
        setc(o.alpha, rnd(st, al));
        o.kappa = kap(h, st);
        setc(o.beta, rnd(st, 1.0 / eta[k - 1]));
        setc(o.gamma, rnd(st, 1.0 / eta[k]));
        o.dot = false;
        if (int rc = do_outer(h, ws, o, ns)) return rc;
        Wcur = Wnxt;
        Wnxt = (Wcur == ws.w[2]) ? ws.w[3] : ws.w[2];
    }
    // x = p_in(A) y; y lives in ws.y which chain_apply_single does not touch
    return chain_apply_single(h, ws, th, ws.y, X);
}

int apply_A(mpmc_ctx* h, Workspace& ws, const void* in, void* out) {
    StepArgs a{};
    a.in = in;
    a.out = out;
    a.op_only = true;
    a.kappa = kap(h, ws.storage);
    const NoiseSpec ns{0, 0, 0};
    return do_step(h, ws, a, ns);
}

int default_nb(const mpmc_ctx* h) {
    if (h->nb_user > 0) return h->nb_user;
    // keep the six work vectors within ~24 GB
    const size_t per = (size_t)h->g.V * 12 * storage_bytes(h->storage) * 6;
    int nb = 64;
    while (nb > 1 && per * nb > (size_t)24 << 30) nb /= 2;
    return nb;
}

int ensure_io(mpmc_ctx* h, size_t ncplx) {
    if (h->io_cap >= ncplx) return MPMC_OK;
    dev_free(h->io);
    h->io_cap = 0;
    if (int rc = dev_alloc(h, &h->io, ncplx * 16)) return rc;
    h->io_cap = ncplx;
    return MPMC_OK;
}

int ensure_defl_work(mpmc_ctx* h, int nb) {
    if (h->k == 0) return MPMC_OK;
    if (h->defl_nb == nb) return MPMC_OK;
    dev_free(h->defl_part);
    dev_free(h->G1);
    dev_free(h->G2);
    dev_free(h->dterm);
    dev_free(h->D);
    dev_free(h->xz);
    const int ns = defl_nsplit(h->g.V);
    if (int rc = dev_alloc(h, &h->defl_part, sizeof(double2) * 2 * (size_t)ns * h->k * nb)) return rc;
    if (int rc = dev_alloc(h, &h->G1, sizeof(double2) * (size_t)h->k * nb)) return rc;
    if (int rc = dev_alloc(h, &h->G2, sizeof(double2) * (size_t)h->k * nb)) return rc;
    if (int rc = dev_alloc(h, &h->dterm, sizeof(double2) * nb)) return rc;
    if (int rc = dev_alloc(h, &h->D, sizeof(double2) * (size_t)h->k * nb)) return rc;
    dev_free(h->D32);
    if (int rc = dev_alloc(h, &h->D32, sizeof(float2) * (size_t)h->k * nb)) return rc;
    if (int rc = dev_alloc(h, &h->xz, sizeof(double2) * nb)) return rc;
    h->defl_nb = nb;
    return MPMC_OK;
}

int level_coefficients(mpmc_ctx* h, int level, std::vector<cd>& c) {
    const int L = num_levels(h);
    c.assign(h->k, 0.0);
    if (h->k == 0 || level >= L - 1) return MPMC_OK;
    for (int i = 0; i < h->k; ++i) {
        c[i] = spec_value(h->polys[level], h->lam[i]) - spec_value(h->polys[level + 1], h->lam[i]);
        if (!finite(c[i])) return fail(h, MPMC_ENONFINITE, "non-finite deflation coefficient");
    }
    return MPMC_OK;
}

void free_deflation(mpmc_ctx* h) {
    dev_free(h->Z);
    dev_free(h->d_pair);
    dev_free(h->d_dnorm);
    dev_free(h->d_coef);
    dev_free(h->AZ);
    dev_free(h->d_Hinv);
    dev_free(h->defl_part);
    dev_free(h->G1);
    dev_free(h->G2);
    dev_free(h->dterm);
    dev_free(h->D);
    dev_free(h->xz);
    dev_free(h->planes);
    dev_free(h->tc_part);
    dev_free(h->D32);
    dev_free(h->Zb);
    dev_free(h->Wb);
    dev_free(h->d_invd);
    dev_free(h->gram_part);
    h->gram_part_cap = 0;
    h->proj_ready = false;
    h->tc_part_cap = 0;
    h->tc_ready = false;
    h->defl_nb = 0;
    h->k = 0;
    h->lam.clear();
    h->pair.clear();
    h->dnorm.clear();
}

int upload_coefficients(mpmc_ctx* h) {
    if (h->k == 0) return MPMC_OK;
    std::vector<double2> all((size_t)MPMC_MAX_POLYS * h->k, make_double2(0, 0));
    const int L = num_levels(h);
    for (int l = 0; l + 1 < L; ++l) {
        std::vector<cd> c;
        if (int rc = level_coefficients(h, l, c)) return rc;
        for (int i = 0; i < h->k; ++i) {
            const cd q = c[i] / h->dnorm[i];
            all[(size_t)l * h->k + i] = make_double2(q.real(), q.imag());
        }
    }
    CK(cudaMemcpyAsync(h->d_coef, all.data(), sizeof(double2) * all.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPMC_OK;
}


// ------------------------------------------------------------------ projected composite (Sec. 4.3)
// In-place inverse of a k x k complex matrix (Gauss-Jordan, partial pivoting).
bool invert(std::vector<cd>& a, int k) {
    std::vector<cd> inv((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) inv[(size_t)i * k + i] = 1.0;
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int r = c + 1; r < k; ++r)
            if (std::abs(a[(size_t)r * k + c]) > std::abs(a[(size_t)piv * k + c])) piv = r;
        if (!(std::abs(a[(size_t)piv * k + c]) > 0)) return false;
        if (piv != c)
            for (int j = 0; j < k; ++j) {
                std::swap(a[(size_t)piv * k + j], a[(size_t)c * k + j]);
                std::swap(inv[(size_t)piv * k + j], inv[(size_t)c * k + j]);
            }
        const cd d = 1.0 / a[(size_t)c * k + c];
        for (int j = 0; j < k; ++j) {
            a[(size_t)c * k + j] *= d;
            inv[(size_t)c * k + j] *= d;
        }
        for (int r = 0; r < k; ++r) {
            if (r == c) continue;
            const cd f = a[(size_t)r * k + c];
            if (f == 0.0) continue;
            for (int j = 0; j < k; ++j) {
                a[(size_t)r * k + j] -= f * a[(size_t)c * k + j];
                inv[(size_t)r * k + j] -= f * inv[(size_t)c * k + j];
            }
        }
    }
    a.swap(inv);
    return true;
}

// Arithmetic of the projection of the projected composite (Sec. 4.3): the handle's math precision.
// (FP64 on reduced-precision handles was measured: r = b - (A Z) D costs k complex FP64 multiply-adds
// per site and vector, 106 ms per 32-vector block at 24^3 x 32 with k = 92 on GB300's FP64 units,
// 7.6 % of a step, and it left the FP32 level estimates unchanged.)
int proj_math(const mpmc_ctx* h) { return h->storage == ST_F64 ? ST_F64 : ST_F32; }

int ensure_gram_part(mpmc_ctx* h, size_t entries) {
    if (h->gram_part_cap >= entries) return MPMC_OK;
    dev_free(h->gram_part);
    h->gram_part_cap = 0;
    if (int rc = dev_alloc(h, &h->gram_part, sizeof(double2) * entries)) return rc;
    h->gram_part_cap = entries;
    return MPMC_OK;
}

// Z and W = A Z in block layout, H = U^H W inverted, 1/d_i: everything the
// projection needs, formed once per deflation set and gauge field.
int ensure_projection(mpmc_ctx* h) {
    if (h->proj_ready) return MPMC_OK;
    if (h->k == 0) return fail(h, MPMC_ESTATE, "the projected composite needs deflation vectors");
    const int k = h->k, math = proj_math(h);
    const size_t bytes = (size_t)nsites12(h) * k * (math == ST_F64 ? 16 : 8);
    dev_free(h->Zb);
    dev_free(h->Wb);
    dev_free(h->d_invd);
    dev_free(h->d_Hinv);
    if (int rc = dev_alloc(h, &h->Zb, bytes)) return rc;
    if (int rc = dev_alloc(h, &h->Wb, bytes)) return rc;
    launch_vec_to_block(math, h->g.V, k, h->Z, h->Zb, h->stream, h->storage == ST_F64 ? ST_F64 : ST_F32);
    LAUNCHED(1);
    StepArgs a{};
    a.in = h->Zb;
    a.out = h->Wb;
    a.op_only = true;
    a.kappa = kap(h, math);
    const NoiseSpec ns0{0, 0, 0};
    launch_step(math, h->g, links_for(h, math), k, ns0, a, chain_config(h->g, k, 64, 1, 1), h->stream);
    LAUNCHED(1);
    const int nsplit = gram_nsplit(h->g.V);
    if (int rc = ensure_gram_part(h, (size_t)nsplit * k * k + (size_t)k * k)) return rc;
    double2* G = h->gram_part + (size_t)nsplit * k * k;
    launch_block_gram(math, h->g.V, h->Zb, k, math, h->Wb, k, 1, h->gram_part, nsplit, G, h->stream);
    LAUNCHED(2);
    std::vector<double2> g((size_t)k * k);
    CK(cudaMemcpyAsync(g.data(), G, sizeof(double2) * g.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // H_ij = u_i^H W_j = (z_pair(i)^H gamma5 W_j) / d_i
    std::vector<cd> H((size_t)k * k);
    std::vector<double2> invd(k);
    for (int i = 0; i < k; ++i) {
        const cd di = 1.0 / h->dnorm[i];
        invd[i] = make_double2(di.real(), di.imag());
        for (int j = 0; j < k; ++j) {
            const double2 v = g[(size_t)h->pair[i] * k + j];
            H[(size_t)i * k + j] = cd(v.x, v.y) * di;
        }
    }
    if (!invert(H, k)) return fail(h, MPMC_ENONFINITE, "U^H A Z is singular");
    std::vector<double2> hinv((size_t)k * k);
    for (size_t q = 0; q < hinv.size(); ++q) {
        if (!finite(H[q])) return fail(h, MPMC_ENONFINITE, "(U^H A Z)^{-1} is not finite");
        hinv[q] = make_double2(H[q].real(), H[q].imag());
    }
    if (int rc = dev_alloc(h, &h->d_Hinv, sizeof(double2) * hinv.size())) return rc;
    if (int rc = dev_alloc(h, &h->d_invd, sizeof(double2) * k)) return rc;
    CK(cudaMemcpyAsync(h->d_Hinv, hinv.data(), sizeof(double2) * hinv.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->d_invd, invd.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->proj_ready = true;
    return MPMC_OK;
}

// G1 = Z^H b, G2 = Z^H gamma5 b for the noise block (tensor or CUDA cores).
int deflation_dots(mpmc_ctx* h, int nb, const NoiseSpec& ns) {
    const bool tcore = h->storage != ST_F64 && h->use_tc && h->tc_ready;
    if (int rc = prof_begin(h, PROF_DEFLATION, (double)h->k * nsites12(h) * (h->storage == ST_F64 ? 16 : 8)))
        return rc;
    if (tcore) {
        int tsplit, kbps;
        size_t pf;
        tc_defl_plan(h->g.V, h->k, nb, &tsplit, &kbps, &pf);
        if (h->tc_part_cap < pf) {
            dev_free(h->tc_part);
            h->tc_part_cap = 0;
            if (int rc = dev_alloc(h, &h->tc_part, pf * sizeof(float))) return rc;
            h->tc_part_cap = pf;
        }
        if (tc_defl_launch(h->tmap, h->g.V, h->k, nb, ns, h->tc_part, tsplit, kbps, h->G1, h->G2, h->d_err,
                           h->stream))
            return fail(h, MPMC_ECUDA, "tensor-core deflation kernel setup failed");
        if (int rc = prof_end(h)) return rc;
        LAUNCHED(2);
    } else {
        const int nsplit = defl_nsplit(h->g.V);
        launch_defl_dots(h->storage == ST_F64 ? ST_F64 : ST_F32, h->g, h->k, h->Z, nb, ns, h->defl_part, nsplit,
                         h->stream);
        if (int rc = prof_end(h)) return rc;
        launch_defl_reduce(h->k, nb, nsplit, h->defl_part, h->d_coef, h->d_pair, h->G1, h->G2, h->dterm, h->stream);
        LAUNCHED(3);
    }
    return MPMC_OK;
}
}  // namespace

// ==================================================================== C ABI
extern "C" {

const char* mpmc_strerror(int code) {
    switch (code) {
        case MPMC_OK: return "ok";
        case MPMC_EINVAL: return "invalid argument";
        case MPMC_ENOMEM: return "out of memory";
        case MPMC_ENOTSUP: return "not supported";
        case MPMC_ETIMEOUT: return "device wait timed out";
        case MPMC_ENONFINITE: return "non-finite value";
        case MPMC_ECUDA: return "CUDA error";
        case MPMC_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

const char* mpmc_last_error(mpmc_handle h) { return h ? h->err.c_str() : "null handle"; }

long long mpmc_launch_count(mpmc_handle h) { return h ? h->launches : 0; }

int mpmc_create(mpmc_handle* out, const int dims[4], const double* links, double kappa, int precision, int bc_t) {
    if (!out) return MPMC_EINVAL;
    *out = nullptr;
    if (!dims || !links) return MPMC_EINVAL;
    for (int d = 0; d < 4; ++d)
        if (dims[d] < 2 || dims[d] > 4096) return MPMC_EINVAL;
    if (!std::isfinite(kappa)) return MPMC_EINVAL;
    if (bc_t != 1 && bc_t != -1) return MPMC_EINVAL;
    if (precision != MPMC_FP64 && precision != MPMC_FP32 && precision != MPMC_BF16S) return MPMC_ENOTSUP;
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V * 12 > (1LL << 31) - 1) return MPMC_EINVAL;
    mpmc_ctx* h = new (std::nothrow) mpmc_ctx();
    if (!h) return MPMC_ENOMEM;
    h->g.lx = dims[0]; h->g.ly = dims[1]; h->g.lz = dims[2]; h->g.lt = dims[3];
    h->g.V = (int)V;
    h->g.bc_t = bc_t;
    h->kappa = kappa;
    h->prec = precision;
    h->storage = precision == MPMC_FP64 ? ST_F64 : (precision == MPMC_FP32 ? ST_F32 : ST_BF16);
    int rc = MPMC_OK;
    auto bail = [&](int code) { mpmc_destroy(h); return code; };
    if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        return bail(MPMC_ECUDA);
    }
    h->stream = h->own;
    const size_t nl = (size_t)V * 36;   // complex link entries
    double* staging = nullptr;
    if ((rc = dev_alloc(h, &staging, nl * 16))) return bail(rc);
    if (cudaMemcpy(staging, links, nl * 16, cudaMemcpyHostToDevice) != cudaSuccess) {
        dev_free(staging);
        return bail(MPMC_ECUDA);
    }
    if ((rc = dev_alloc(h, &h->d_err, sizeof(int)))) { dev_free(staging); return bail(rc); }
    if (cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess) { dev_free(staging); return bail(MPMC_ECUDA); }
    if ((rc = dev_alloc(h, &h->links64, nl * 16))) { dev_free(staging); return bail(rc); }
    launch_links(ST_F64, h->g.V, staging, h->links64, h->stream);
    if (h->storage != ST_F64) {
        if ((rc = dev_alloc(h, &h->links32, nl * 8))) { dev_free(staging); return bail(rc); }
        launch_links(ST_F32, h->g.V, staging, h->links32, h->stream, h->kappa);
        if ((rc = dev_alloc(h, &h->links_ex, nl * 16))) { dev_free(staging); return bail(rc); }
        launch_links_expanded(h->g.V, staging, h->links_ex, h->stream, h->kappa);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        dev_free(staging);
        return bail(MPMC_ECUDA);
    }
    dev_free(staging);
    *out = h;
    return MPMC_OK;
}

int mpmc_destroy(mpmc_handle h) {
    if (!h) return MPMC_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_ws(h->ws);
    free_ws(h->ws64);
    free_deflation(h);
    dev_free(h->links64);
    dev_free(h->links32);
    dev_free(h->links_ex);
    dev_free(h->probe);
    dev_free(h->probe_tab);
    dev_free(h->blk_order);
    dev_free(h->sol);
    dev_free(h->samples);
    dev_free(h->io);
    dev_free(h->kr_part);
    dev_free(h->kr_h);
    dev_free(h->kr_nrm);
    dev_free(h->d_err);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->own) cudaStreamDestroy(h->own);
    delete h;
    return MPMC_OK;
}

int mpmc_set_stream(mpmc_handle h, void* stream) {
    if (h) ++h->gen;
    if (!h) return MPMC_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    h->stream = stream ? (cudaStream_t)stream : h->own;
    return MPMC_OK;
}

int mpmc_set_block(mpmc_handle h, int nb) {
    if (h) ++h->gen;
    if (!h) return MPMC_EINVAL;
    if (nb < 0 || nb > MPMC_MAX_BLOCK) return fail(h, MPMC_EINVAL, "block size out of range");
    h->nb_user = nb;
    return MPMC_OK;
}

int mpmc_set_poly(mpmc_handle h, int index, int kind, const double* roots, int nroots, const double* outer,
                  int nouter, int leja) {
    if (h) ++h->gen;
    if (!h) return MPMC_EINVAL;
    if (index < 0 || index >= MPMC_MAX_POLYS) return fail(h, MPMC_EINVAL, "polynomial index out of range");
    if (kind != MPMC_SINGLE && kind != MPMC_COMPOSITE && kind != MPMC_DEFLATED_COMPOSITE)
        return fail(h, MPMC_EINVAL, "unknown polynomial kind");
    if (!roots || nroots < 1 || nroots > 100000) return fail(h, MPMC_EINVAL, "need at least one root");
    if (kind != MPMC_SINGLE && (!outer || nouter < 1 || nouter > 100000))
        return fail(h, MPMC_EINVAL, "composite polynomial needs outer roots");
    if (kind == MPMC_DEFLATED_COMPOSITE && h->k == 0)
        return fail(h, MPMC_ESTATE, "projected composite needs mpmc_set_deflation first");
    if (kind == MPMC_DEFLATED_COMPOSITE && index != 0)
        return fail(h, MPMC_EINVAL, "the projected composite can only be polynomial 0 (the highest level)");
    if (kind == MPMC_DEFLATED_COMPOSITE && nouter < 2)
        return fail(h, MPMC_EINVAL, "projected composite needs at least two outer roots");
    PolyDef p;
    p.kind = kind;
    for (int i = 0; i < nroots; ++i) p.roots.emplace_back(roots[2 * i], roots[2 * i + 1]);
    if (kind != MPMC_SINGLE)
        for (int i = 0; i < nouter; ++i) p.outer.emplace_back(outer[2 * i], outer[2 * i + 1]);
    for (const cd& z : p.roots)
        if (!finite(z) || z == 0.0) return fail(h, MPMC_ENONFINITE, "root is zero or not finite");
    for (const cd& z : p.outer)
        if (!finite(z) || z == 0.0) return fail(h, MPMC_ENONFINITE, "outer root is zero or not finite");
    if (leja & MPMC_POLY_FP32_COEFS) {
        // theta -> 1 / fl32(1 / theta): the coefficient every precision applies is an FP32 number
        auto snap = [](cd z) {
            const cd c = 1.0 / z;
            return 1.0 / cd((double)(float)c.real(), (double)(float)c.imag());
        };
        for (cd& z : p.roots) z = snap(z);
        for (cd& z : p.outer) z = snap(z);
        for (const cd& z : p.roots)
            if (!finite(z)) return fail(h, MPMC_ENONFINITE, "root outside the FP32 range");
        for (const cd& z : p.outer)
            if (!finite(z)) return fail(h, MPMC_ENONFINITE, "outer root outside the FP32 range");
    }
    if (leja & MPMC_POLY_LEJA) {
        auto o = leja_order(p.roots);
        std::vector<cd> r(p.roots.size());
        for (size_t i = 0; i < o.size(); ++i) r[i] = p.roots[o[i]];
        p.roots.swap(r);
        if (!p.outer.empty()) {
            auto oo = leja_order(p.outer);
            std::vector<cd> q(p.outer.size());
            for (size_t i = 0; i < oo.size(); ++i) q[i] = p.outer[oo[i]];
            p.outer.swap(q);
        }
    }
    p.set = true;
    h->polys[index] = p;
    return upload_coefficients(h);
}

int mpmc_get_roots(mpmc_handle h, int index, double* roots, double* outer) {
    if (!h) return MPMC_EINVAL;
    if (index < 0 || index >= MPMC_MAX_POLYS) return fail(h, MPMC_EINVAL, "polynomial index out of range");
    const PolyDef& p = h->polys[index];
    if (!p.set) return fail(h, MPMC_ESTATE, "polynomial not set");
    if (roots)
        for (size_t i = 0; i < p.roots.size(); ++i) { roots[2 * i] = p.roots[i].real(); roots[2 * i + 1] = p.roots[i].imag(); }
    if (outer)
        for (size_t i = 0; i < p.outer.size(); ++i) { outer[2 * i] = p.outer[i].real(); outer[2 * i + 1] = p.outer[i].imag(); }
    return MPMC_OK;
}

static int set_deflation_impl(mpmc_handle h, const double* Z, const double* lambda, const int* pair, int k,
                              int on_device) {
    if (!h) return MPMC_EINVAL;
    const long long n = nsites12(h);
    if (k < 0 || k > n || k > 4096) return fail(h, MPMC_EINVAL, "k out of range");
    CK(cudaStreamSynchronize(h->stream));
    free_deflation(h);
    for (int p = 0; p < MPMC_MAX_POLYS; ++p)
        if (h->polys[p].set && h->polys[p].kind == MPMC_DEFLATED_COMPOSITE && k == 0)
            return fail(h, MPMC_ESTATE, "a projected composite polynomial needs deflation vectors");
    if (k == 0) return MPMC_OK;
    if (!Z || !lambda || !pair) return fail(h, MPMC_EINVAL, "null deflation input");
    for (int i = 0; i < k; ++i) {
        if (pair[i] < 0 || pair[i] >= k) return fail(h, MPMC_EINVAL, "pair index out of range");
        if (pair[pair[i]] != i) return fail(h, MPMC_EINVAL, "pair map is not an involution");
        if (!std::isfinite(lambda[2 * i]) || !std::isfinite(lambda[2 * i + 1]) ||
            (lambda[2 * i] == 0 && lambda[2 * i + 1] == 0))
            return fail(h, MPMC_ENONFINITE, "eigenvalue is zero or not finite");
    }
    h->k = k;
    for (int i = 0; i < k; ++i) h->lam.emplace_back(lambda[2 * i], lambda[2 * i + 1]);
    h->pair.assign(pair, pair + k);
    const size_t ncplx = (size_t)n * k;
    const int zst = h->storage == ST_F64 ? ST_F64 : ST_F32;
    if (int rc = ensure_io(h, ncplx)) return rc;
    CK(cudaMemcpyAsync(h->io, Z, ncplx * 16, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream));
    if (int rc = dev_alloc(h, &h->Z, ncplx * (zst == ST_F64 ? 16 : 8))) return rc;
    if (zst == ST_F64) {
        launch_convert_vectors(zst, ncplx, h->io, h->Z, h->stream);
        LAUNCHED(1);
    } else {
        // reduced precision: z is held as zhat = hi + lo (two BF16 terms, exact in FP32); the
        // CUDA-core and tensor-core dots and the exact correction all use these same vectors
        int Mpad, Kpad;
        tc_defl_layout(h->g.V, k, &Mpad, &Kpad);
        if (int rc = dev_alloc(h, &h->planes, (size_t)2 * Mpad * Kpad * 2)) return rc;
        launch_split_bf16(h->g.V, k, Mpad, Kpad, h->io, reinterpret_cast<float*>(h->Z), h->planes, h->stream);
        LAUNCHED(1);
        h->tc_ready = tc_make_map(h->tmap, h->planes, Mpad, Kpad);
    }
    if (int rc = dev_alloc(h, &h->d_pair, sizeof(int) * k)) return rc;
    CK(cudaMemcpyAsync(h->d_pair, pair, sizeof(int) * k, cudaMemcpyHostToDevice, h->stream));
    if (int rc = dev_alloc(h, &h->d_dnorm, sizeof(double2) * k)) return rc;
    launch_defl_norms(zst, h->g.V, k, h->Z, h->d_pair, h->d_dnorm, h->stream);
    LAUNCHED(1);
    std::vector<double2> dn(k);
    CK(cudaMemcpyAsync(dn.data(), h->d_dnorm, sizeof(double2) * k, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < k; ++i) {
        h->dnorm.emplace_back(dn[i].x, dn[i].y);
        if (!finite(h->dnorm[i]) || h->dnorm[i] == 0.0)
            return fail(h, MPMC_ENONFINITE, "u_i^H z_i is zero or not finite");
    }
    if (int rc = dev_alloc(h, &h->d_coef, sizeof(double2) * (size_t)MPMC_MAX_POLYS * k)) return rc;
    return upload_coefficients(h);
}

}  // extern "C"

namespace {

// Sum of v^H p(A) v over the 12 * ncolours probe vectors of a colouring: from the device
// table tab (V entries) or, with tab == nullptr, the period-m colouring.
int probing_sum(mpmc_ctx* h, int index, int m, const int* tab, long long ncolours, double* trace) {
    if (!trace) return fail(h, MPMC_EINVAL, "trace is NULL");
    if (index < 0 || index >= MPMC_MAX_POLYS) return fail(h, MPMC_EINVAL, "polynomial index out of range");
    const PolyDef& p = h->polys[index];
    if (!p.set) return fail(h, MPMC_ESTATE, "polynomial not set");
    if (p.kind == MPMC_DEFLATED_COMPOSITE) return fail(h, MPMC_ENOTSUP, "probing of the projected composite");
    const long long nq_all = 12LL * ncolours;
    const int nb = (int)std::min<long long>(default_nb(h), nq_all);
    if (int rc = ensure_ws(h, h->ws, h->storage, nb)) return rc;
    const int nchunk = 152;
    const size_t need = (size_t)nchunk * nb + 1;
    if (h->probe_cap < need) {
        dev_free(h->probe);
        h->probe_cap = 0;
        if (int rc = dev_alloc(h, &h->probe, sizeof(double2) * need)) return rc;
        h->probe_cap = need;
    }
    double2* total = h->probe + (size_t)nchunk * nb;
    CK(cudaMemsetAsync(total, 0, sizeof(double2), h->stream));
    Workspace& ws = h->ws;
    for (long long q0 = 0; q0 < nq_all; q0 += nb) {
        const int cnt = (int)std::min<long long>(nb, nq_all - q0);
        launch_probe_block(ws.storage, h->g, m, tab, (int)q0, cnt, nb, ws.r, h->stream);
        LAUNCHED(1);
        if (int rc = chain_apply(h, ws, p, ws.r, ws.x)) return rc;
        launch_probe_trace(ws.storage, h->g, m, tab, (int)q0, cnt, nb, ws.x, nchunk, h->probe, total, h->stream);
        LAUNCHED(2);
    }
    double2 t;
    CK(cudaMemcpyAsync(&t, total, sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (int rc = device_flag(h)) return rc;
    trace[0] = t.x;
    trace[1] = t.y;
    return prof_collect(h);
}

}  // namespace

extern "C" {

int mpmc_trace_probing(mpmc_handle h, int index, int m, double* trace) {
    if (!h) return MPMC_EINVAL;
    if (m < 1 || h->g.lx % m || h->g.ly % m || h->g.lz % m || h->g.lt % m)
        return fail(h, MPMC_EINVAL, "the period m must divide every lattice extent");
    return probing_sum(h, index, m, nullptr, 1LL * m * m * m * m, trace);
}

int mpmc_trace_probing_colours(mpmc_handle h, int index, const int* colours, int ncolours, double* trace) {
    if (!h) return MPMC_EINVAL;
    if (!colours || ncolours < 1 || ncolours > h->g.V) return fail(h, MPMC_EINVAL, "bad colouring");
    for (int s = 0; s < h->g.V; ++s)
        if (colours[s] < 0 || colours[s] >= ncolours) return fail(h, MPMC_EINVAL, "a site colour is out of range");
    if ((size_t)h->g.V > h->probe_tab_cap) {
        dev_free(h->probe_tab);
    dev_free(h->blk_order);
        h->probe_tab_cap = 0;
        if (int rc = dev_alloc(h, &h->probe_tab, sizeof(int) * (size_t)h->g.V)) return rc;
        h->probe_tab_cap = h->g.V;
    }
    CK(cudaMemcpyAsync(h->probe_tab, colours, sizeof(int) * (size_t)h->g.V, cudaMemcpyHostToDevice, h->stream));
    return probing_sum(h, index, 1, h->probe_tab, ncolours, trace);
}

// ------------------------------------------------------------------ linear equations
// Right-preconditioned restarted GMRES(m) for A x = b with the operator A p_in(A) (Sec. 2.4:
// polynomial preconditioning; pin < 0: plain GMRES), FP64, one right-hand side, and a
// Left-right Projection with the deflation vectors before every cycle (Secs. 2.1, 5 step 3a):
// x += Z H^{-1} U^H r, r -= A Z H^{-1} U^H r.  b, x: n complex on the device.
int solve_one(mpmc_ctx* h, int pin, const double2* b, double2* x, double rtol, int m, int maxcycles, double* relres,
              long long* matvecs) {
    const size_t n = nsites12(h);
    Workspace& ws = h->ws64;
    // solver area: basis V (m+1 vectors), r, t, u, then two caller vectors (b, x), then coefficients
    double2* Vb = h->sol;
    double2* r = Vb + (size_t)(m + 1) * n;
    double2* t = r + n;
    double2* u = t + n;
    double2* coef = u + 3 * n;       // m + 2 device coefficients
    double* part = reinterpret_cast<double*>(h->kr_part);
    double* nrm = h->kr_nrm;
    const bool defl = h->k > 0;
    const long long mv_pin = pin >= 0 ? spec_matvecs(h->polys[pin]) + 1 : 1;
    auto norm = [&](const double2* v, double* out) -> int {
        launch_norm2(n, v, part, nrm, h->stream);
        LAUNCHED(1);
        double nn = 0;
        CK(cudaMemcpyAsync(&nn, nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        *out = std::sqrt(nn);
        return MPMC_OK;
    };
    auto set_coef = [&](const std::vector<double2>& c) -> int {
        CK(cudaMemcpyAsync(coef, c.data(), sizeof(double2) * c.size(), cudaMemcpyHostToDevice, h->stream));
        return MPMC_OK;
    };
    // op(v) -> out:  A p_in(A) v  (p_in(A) v left in t when pin >= 0)
    auto op = [&](const double2* v, double2* out) -> int {
        const double2* in = v;
        if (pin >= 0) {
            if (int e = chain_apply(h, ws, h->polys[pin], v, t)) return e;
            in = t;
        }
        return apply_A(h, ws, in, out);
    };
    double bn = 0;
    if (int e = norm(b, &bn)) return e;
    CK(cudaMemsetAsync(x, 0, n * 16, h->stream));
    *matvecs = 0;
    double rn = bn;
    for (int cycle = 0; cycle <= maxcycles; ++cycle) {
        // r = b - A x
        if (int e = apply_A(h, ws, x, u)) return e;
        ++*matvecs;
        CK(cudaMemcpyAsync(r, b, n * 16, cudaMemcpyDeviceToDevice, h->stream));
        if (int e = set_coef({make_double2(1.0, 0.0)})) return e;
        launch_maxpy(n, 1, u, coef, r, h->stream);
        LAUNCHED(1);
        if (defl) {
            const int nsplit = gram_nsplit(h->g.V);
            if (int e = ensure_gram_part(h, (size_t)nsplit * h->k)) return e;
            launch_block_gram(ST_F64, h->g.V, h->Zb, h->k, ST_F64, r, 1, 1, h->gram_part, nsplit, h->G2, h->stream);
            launch_proj_coef(h->k, 1, h->d_pair, h->d_invd, h->d_Hinv, nullptr, h->G2, h->D, h->D32, nullptr,
                             h->stream);
            launch_rank_update(ST_F64, ST_F64, h->g.V, 1, h->Zb, h->k, h->D, h->D32, 1.0, x, NoiseSpec{0, 0, 0}, x,
                               h->stream);
            launch_rank_update(ST_F64, ST_F64, h->g.V, 1, h->Wb, h->k, h->D, h->D32, -1.0, r, NoiseSpec{0, 0, 0}, r,
                               h->stream);
            LAUNCHED(4);
        }
        if (int e = norm(r, &rn)) return e;
        if (!(rn > rtol * bn) || cycle == maxcycles || !std::isfinite(rn)) break;
        // Arnoldi on A p_in(A) from r / |r|, with Givens rotations on the host
        std::vector<cd> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
        g[0] = rn;
        CK(cudaMemsetAsync(Vb, 0, n * 16, h->stream));
        if (int e = set_coef({make_double2(-1.0 / rn, 0.0)})) return e;
        launch_maxpy(n, 1, r, coef, Vb, h->stream);   // V_0 = r / |r|
        LAUNCHED(1);
        std::vector<double2> h1(m + 1), h2(m + 1);
        int j = 0;
        for (; j < m; ++j) {
            double2* vj = Vb + (size_t)j * n;
            double2* w = Vb + (size_t)(j + 1) * n;
            if (int e = op(vj, w)) return e;
            *matvecs += mv_pin;
            launch_mdot(n, j + 1, Vb, w, h->kr_part, h->kr_h, h->stream);
            launch_maxpy(n, j + 1, Vb, h->kr_h, w, h->stream);
            CK(cudaMemcpyAsync(h1.data(), h->kr_h, sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost, h->stream));
            launch_mdot(n, j + 1, Vb, w, h->kr_part, h->kr_h + (m + 1), h->stream);
            launch_maxpy(n, j + 1, Vb, h->kr_h + (m + 1), w, h->stream);
            CK(cudaMemcpyAsync(h2.data(), h->kr_h + (m + 1), sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost,
                               h->stream));
            LAUNCHED(4);
            double beta = 0;
            if (int e = norm(w, &beta)) return e;
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = cd(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
            H[(size_t)(j + 1) * m + j] = beta;
            if (beta > 0 && std::isfinite(beta)) {
                launch_normalize(n, w, nrm, w, h->stream);
                LAUNCHED(1);
            }
            // apply the previous rotations to column j, then a new one
            for (int i = 0; i < j; ++i) {
                const cd a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            const cd a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
            const double den = std::sqrt(std::norm(a) + std::norm(c));
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? c / den : 0.0;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = std::conj(cs[j]) * g[j];
            if (std::abs(g[j + 1]) <= rtol * bn || !(beta > 0)) { ++j; break; }
        }
        // y = R^{-1} g, x += p_in(A) V y
        std::vector<cd> y(j);
        for (int i = j - 1; i >= 0; --i) {
            cd acc = g[i];
            for (int l = i + 1; l < j; ++l) acc -= H[(size_t)i * m + l] * y[l];
            y[i] = acc / H[(size_t)i * m + i];
        }
        std::vector<double2> yc(j);
        for (int i = 0; i < j; ++i) yc[i] = make_double2(y[i].real(), y[i].imag());
        if (int e = set_coef(yc)) return e;
        launch_combine(n, j, Vb, coef, 1, u, h->stream);
        LAUNCHED(1);
        const double2* add = u;
        if (pin >= 0) {
            if (int e = chain_apply(h, ws, h->polys[pin], u, t)) return e;
            *matvecs += mv_pin - 1;
            add = t;
        }
        if (int e = set_coef({make_double2(-1.0, 0.0)})) return e;
        launch_maxpy(n, 1, add, coef, x, h->stream);
        LAUNCHED(1);
    }
    *relres = rn / bn;
    return MPMC_OK;
}

int solve_setup(mpmc_ctx* h, int pin, int m) {
    if (h->storage != ST_F64) return fail(h, MPMC_ENOTSUP, "linear solves run on FP64 handles");
    if (m < 1 || m > 1024) return fail(h, MPMC_EINVAL, "restart length out of range");
    if (pin >= MPMC_MAX_POLYS || (pin >= 0 && !h->polys[pin].set)) return fail(h, MPMC_ESTATE, "p_in not set");
    if (pin >= 0 && h->polys[pin].kind != MPMC_SINGLE) return fail(h, MPMC_ENOTSUP, "p_in must be a single polynomial");
    const size_t n = nsites12(h);
    if (int rc = ensure_ws(h, h->ws64, ST_F64, 1)) return rc;
    const size_t need = (size_t)(m + 6) * n + (m + 2);
    if (h->sol_cap < need) {
        dev_free(h->sol);
        h->sol_cap = 0;
        if (int rc = dev_alloc(h, &h->sol, sizeof(double2) * need)) return rc;
        h->sol_cap = need;
    }
    if (h->kr_m < m + 1) {
        dev_free(h->kr_part);
        dev_free(h->kr_h);
        dev_free(h->kr_nrm);
        h->kr_m = 0;
        const int np = mdot_parts(n);
        if (int rc = dev_alloc(h, &h->kr_part, sizeof(double2) * (size_t)np * (m + 1))) return rc;
        if (int rc = dev_alloc(h, &h->kr_h, sizeof(double2) * 2 * (m + 1))) return rc;
        if (int rc = dev_alloc(h, &h->kr_nrm, sizeof(double) * (np + 1))) return rc;
        h->kr_m = m + 1;
    }
    if (h->k > 0) {
        if (int rc = ensure_defl_work(h, 1)) return rc;
        if (int rc = ensure_projection(h)) return rc;
    }
    return MPMC_OK;
}

int mpmc_solve(mpmc_handle h, int pin, const double* B, double* X, int nrhs, double rtol, int m, int maxcycles,
               int on_device, double* relres, long long* matvecs) {
    if (!h) return MPMC_EINVAL;
    if (!B || !X || nrhs < 1 || !(rtol > 0) || maxcycles < 0) return fail(h, MPMC_EINVAL, "bad solve arguments");
    if (int rc = solve_setup(h, pin, m)) return rc;
    const size_t n = nsites12(h);
    const double* src = B;
    double* dst = X;
    if (!on_device) {
        if (int rc = ensure_io(h, n * nrhs)) return rc;
        CK(cudaMemcpyAsync(h->io, B, n * nrhs * 16, cudaMemcpyHostToDevice, h->stream));
        src = h->io;
        dst = h->io;
    }
    double2* b = h->sol + (size_t)(m + 4) * n;
    double2* x = b + n;
    long long total_mv = 0;
    for (int c = 0; c < nrhs; ++c) {
        launch_import(ST_F64, h->g.V, src, nrhs, c, 1, b, 1, h->stream);
        LAUNCHED(1);
        double rr = 0;
        long long mv = 0;
        if (int rc = solve_one(h, pin, b, x, rtol, m, maxcycles, &rr, &mv)) return rc;
        if (relres) relres[c] = rr;
        total_mv += mv;
        launch_export(ST_F64, h->g.V, x, 1, dst, nrhs, c, 1, h->stream);
        LAUNCHED(1);
    }
    if (!on_device) CK(cudaMemcpyAsync(X, h->io, n * nrhs * 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (matvecs) *matvecs = total_mv;
    return device_flag(h);
}

int mpmc_trace_inverse(mpmc_handle h, int p1, int pin, uint64_t seed, int nsamples, int first, double rtol, int m,
                       int maxcycles, double* mean, double* var, double* samples) {
    if (!h) return MPMC_EINVAL;
    if (nsamples < 1 || first < 0 || !(rtol > 0)) return fail(h, MPMC_EINVAL, "bad trace_inverse arguments");
    if (p1 < 0 || p1 >= MPMC_MAX_POLYS || !h->polys[p1].set) return fail(h, MPMC_ESTATE, "p_1 not set");
    const bool proj = h->polys[p1].kind == MPMC_DEFLATED_COMPOSITE;
    if (proj && h->k == 0) return fail(h, MPMC_ESTATE, "the projected composite needs deflation vectors");
    if (int rc = solve_setup(h, pin, m)) return rc;
    const size_t n = nsites12(h);
    const int k = h->k;
    Workspace& ws = h->ws64;
    // c_i = 1/lambda_i - p_1(lambda_i), divided by d_i for the stored left vectors
    std::vector<cd> c(k);
    cd corr = 0.0;
    for (int i = 0; i < k; ++i) {
        c[i] = 1.0 / h->lam[i] - spec_value(h->polys[p1], h->lam[i]);
        corr += c[i];   // sum_i c_i u_i^H z_i with u_i^H z_i = 1
    }
    std::vector<cd> s(nsamples);
    double2* b = h->sol + (size_t)(m + 4) * n;          // solver area (see solve_one)
    double2* x = b + n;
    double2* pb = h->sol + (size_t)(m + 3) * n;         // u: free between solves
    std::vector<double2> g1(k > 0 ? k : 1), g2(k > 0 ? k : 1);
    double2 dot;
    for (int j = 0; j < nsamples; ++j) {
        const NoiseSpec ns{seed, 0xFFFFu, (uint32_t)(first + j)};
        launch_noise_f64(h->g, ns, 1, 1, 0, reinterpret_cast<double*>(b), h->stream);
        LAUNCHED(1);
        double rr = 0;
        long long mv = 0;
        if (int rc = solve_one(h, pin, b, x, rtol, m, maxcycles, &rr, &mv)) return rc;
        // b^H x
        launch_mdot(n, 1, b, x, h->kr_part, h->kr_h, h->stream);
        CK(cudaMemcpyAsync(&dot, h->kr_h, sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        cd sample(dot.x, dot.y);
        // b^H p_1(A) b;  projected p_1 (Sec. 4.3): M_1 b = Z D + p_1(A)(b - (A Z) D), D = H^{-1} U^H b
        if (proj) {
            double2* r = h->sol + (size_t)(m + 1) * n;      // the solver's residual: free between solves
            const int nsplit = gram_nsplit(h->g.V);
            if (int rc = ensure_gram_part(h, (size_t)nsplit * k)) return rc;
            launch_block_gram(ST_F64, h->g.V, h->Zb, k, ST_F64, b, 1, 1, h->gram_part, nsplit, h->G2, h->stream);
            launch_proj_coef(k, 1, h->d_pair, h->d_invd, h->d_Hinv, nullptr, h->G2, h->D, h->D32, nullptr,
                             h->stream);
            launch_rank_update(ST_F64, ST_F64, h->g.V, 1, h->Wb, k, h->D, h->D32, -1.0, b, NoiseSpec{0, 0, 0}, r,
                               h->stream);
            LAUNCHED(4);
            if (int rc = chain_apply(h, ws, h->polys[p1], r, pb)) return rc;
            launch_rank_update(ST_F64, ST_F64, h->g.V, 1, h->Zb, k, h->D, h->D32, 1.0, pb, NoiseSpec{0, 0, 0}, pb,
                               h->stream);
            LAUNCHED(1);
        } else if (int rc = chain_apply(h, ws, h->polys[p1], b, pb)) {
            return rc;
        }
        launch_mdot(n, 1, b, pb, h->kr_part, h->kr_h, h->stream);
        CK(cudaMemcpyAsync(&dot, h->kr_h, sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
        LAUNCHED(2);
        CK(cudaStreamSynchronize(h->stream));
        sample -= cd(dot.x, dot.y);
        if (k > 0 && !proj) {
            // sum_i c_i (b^H z_i)(u_i^H b), u_i = gamma5 z_pair(i) / conj(d_i)
            const int nsplit = gram_nsplit(h->g.V);
            if (int rc = ensure_gram_part(h, (size_t)nsplit * k)) return rc;
            launch_block_gram(ST_F64, h->g.V, h->Zb, k, ST_F64, b, 1, 0, h->gram_part, nsplit, h->G1, h->stream);
            launch_block_gram(ST_F64, h->g.V, h->Zb, k, ST_F64, b, 1, 1, h->gram_part, nsplit, h->G2, h->stream);
            LAUNCHED(2);
            CK(cudaMemcpyAsync(g1.data(), h->G1, sizeof(double2) * k, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaMemcpyAsync(g2.data(), h->G2, sizeof(double2) * k, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            cd dt = 0.0;
            for (int i = 0; i < k; ++i) {
                const cd bz = std::conj(cd(g1[i].x, g1[i].y));                  // b^H z_i
                const int pi = h->pair[i];
                const cd ub = cd(g2[pi].x, g2[pi].y) / h->dnorm[i];           // u_i^H b
                dt += c[i] * bz * ub;
            }
            sample -= dt;
        }
        if (!std::isfinite(sample.real()) || !std::isfinite(sample.imag()))
            return fail(h, MPMC_ENONFINITE, "non-finite sample");
        s[j] = sample;
    }
    double mr = 0, mi = 0;
    for (const cd& z : s) { mr += z.real(); mi += z.imag(); }
    mr /= nsamples;
    mi /= nsamples;
    double v = NAN;
    if (nsamples > 1) {
        v = 0;
        for (const cd& z : s) v += (z.real() - mr) * (z.real() - mr);
        v /= (nsamples - 1);
    }
    if (mean) { mean[0] = mr + corr.real(); mean[1] = mi + corr.imag(); }
    if (var) *var = v;
    if (samples)
        for (int j = 0; j < nsamples; ++j) { samples[2 * j] = s[j].real(); samples[2 * j + 1] = s[j].imag(); }
    return device_flag(h);
}

int mpmc_deflation_norms(mpmc_handle h, double* d) {
    if (!h) return MPMC_EINVAL;
    if (!d) return fail(h, MPMC_EINVAL, "null output");
    if (h->k == 0) return fail(h, MPMC_ESTATE, "no deflation vectors set");
    for (int i = 0; i < h->k; ++i) {
        d[2 * i] = h->dnorm[i].real();
        d[2 * i + 1] = h->dnorm[i].imag();
    }
    return MPMC_OK;
}

int mpmc_level_info(mpmc_handle h, int level, double* correction, long long* matvecs) {
    if (!h) return MPMC_EINVAL;
    const int L = num_levels(h);
    if (L == 0) return fail(h, MPMC_ESTATE, "no polynomial set");
    if (level < 0 || level >= L) return fail(h, MPMC_EINVAL, "level out of range");
    if (correction) {
        std::vector<cd> c;
        if (int rc = level_coefficients(h, level, c)) return rc;
        cd s = 0.0;
        for (const cd& q : c) s += q;   // u_i^H z_i = 1 by the library's scaling
        correction[0] = s.real();
        correction[1] = s.imag();
    }
    if (matvecs) {
        long long mv = spec_matvecs(h->polys[level]);
        if (level + 1 < L) mv += spec_matvecs(h->polys[level + 1]);
        *matvecs = mv;
    }
    return MPMC_OK;
}

int mpmc_apply_op(mpmc_handle h, const double* X, double* Y, int nrhs, int on_device) {
    if (!h || !X || !Y || nrhs < 1) return h ? fail(h, MPMC_EINVAL, "bad apply_op arguments") : MPMC_EINVAL;
    const size_t n = nsites12(h);
    const int nb = std::min(default_nb(h), nrhs);
    if (int rc = ensure_ws(h, h->ws, h->storage, nb)) return rc;
    const double* src = X;
    double* dst = Y;
    if (!on_device) {
        if (int rc = ensure_io(h, n * nrhs)) return rc;
        CK(cudaMemcpyAsync(h->io, X, n * nrhs * 16, cudaMemcpyHostToDevice, h->stream));
        src = h->io;
        dst = h->io;
    }
    for (int c0 = 0; c0 < nrhs; c0 += nb) {
        const int cnt = std::min(nb, nrhs - c0);
        launch_import(h->storage, h->g.V, src, nrhs, c0, cnt, h->ws.w[2], nb, h->stream);
        LAUNCHED(1);
        if (int rc = apply_A(h, h->ws, h->ws.w[2], h->ws.w[3])) return rc;
        launch_export(h->storage, h->g.V, h->ws.w[3], nb, dst, nrhs, c0, cnt, h->stream);
        LAUNCHED(1);
    }
    if (!on_device) CK(cudaMemcpyAsync(Y, h->io, n * nrhs * 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (int rc = device_flag(h)) return rc;
    return prof_collect(h);
}

int mpmc_apply_poly(mpmc_handle h, int index, const double* B, double* X, int nrhs, int on_device) {
    if (!h) return MPMC_EINVAL;
    if (!B || !X || nrhs < 1) return fail(h, MPMC_EINVAL, "bad apply_poly arguments");
    if (index < 0 || index >= MPMC_MAX_POLYS) return fail(h, MPMC_EINVAL, "polynomial index out of range");
    const PolyDef& p = h->polys[index];
    if (!p.set) return fail(h, MPMC_ESTATE, "polynomial not set");
    const size_t n = nsites12(h);
    const int nb = std::min(default_nb(h), nrhs);
    if (int rc = ensure_ws(h, h->ws, h->storage, nb)) return rc;
    if (p.kind == MPMC_DEFLATED_COMPOSITE) {
        if (int rc = ensure_defl_work(h, nb)) return rc;
        if (int rc = ensure_projection(h)) return rc;
    }
    const double* src = B;
    double* dst = X;
    if (!on_device) {
        if (int rc = ensure_io(h, n * nrhs)) return rc;
        CK(cudaMemcpyAsync(h->io, B, n * nrhs * 16, cudaMemcpyHostToDevice, h->stream));
        src = h->io;
        dst = h->io;
    }
    for (int c0 = 0; c0 < nrhs; c0 += nb) {
        const int cnt = std::min(nb, nrhs - c0);
        launch_import(h->storage, h->g.V, src, nrhs, c0, cnt, h->ws.r, nb, h->stream);
        LAUNCHED(1);
        const bool proj = p.kind == MPMC_DEFLATED_COMPOSITE;
        if (proj) {
            // x = Z D + p_1(A) (B - (A Z) D),  D = H^{-1} U^H B,  U^H B from Z^H gamma5 B
            const int nsplit = gram_nsplit(h->g.V);
            if (int rc = ensure_gram_part(h, (size_t)nsplit * h->k * nb)) return rc;
            launch_block_gram(proj_math(h), h->g.V, h->Zb, h->k, h->storage, h->ws.r, nb, 1, h->gram_part, nsplit,
                              h->G2, h->stream);
            launch_proj_coef(h->k, nb, h->d_pair, h->d_invd, h->d_Hinv, nullptr, h->G2, h->D, h->D32, nullptr,
                             h->stream);
            launch_rank_update(proj_math(h), h->storage, h->g.V, nb, h->Wb, h->k, h->D, h->D32, -1.0, h->ws.r,
                               NoiseSpec{0, 0, 0}, h->ws.r, h->stream);
            LAUNCHED(4);
        }
        if (int rc = chain_apply(h, h->ws, p, h->ws.r, h->ws.x)) return rc;
        if (proj) {
            launch_rank_update(proj_math(h), h->storage, h->g.V, nb, h->Zb, h->k, h->D, h->D32, 1.0, h->ws.x,
                               NoiseSpec{0, 0, 0}, h->ws.x, h->stream);
            LAUNCHED(1);
        }
        launch_export(h->storage, h->g.V, h->ws.x, nb, dst, nrhs, c0, cnt, h->stream);
        LAUNCHED(1);
    }
    if (!on_device) CK(cudaMemcpyAsync(X, h->io, n * nrhs * 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (int rc = device_flag(h)) return rc;
    return prof_collect(h);
}

int mpmc_noise(mpmc_handle h, uint64_t seed, int level, int first, int nrhs, double* B, int on_device) {
    if (!h) return MPMC_EINVAL;
    if (!B || nrhs < 1 || level < 0 || first < 0) return fail(h, MPMC_EINVAL, "bad noise arguments");
    const size_t n = nsites12(h);
    double* dst = B;
    if (!on_device) {
        if (int rc = ensure_io(h, n * nrhs)) return rc;
        dst = h->io;
    }
    NoiseSpec ns{seed, (uint32_t)level, (uint32_t)first};
    launch_noise_f64(h->g, ns, nrhs, nrhs, 0, dst, h->stream);
    LAUNCHED(1);
    if (!on_device) CK(cudaMemcpyAsync(B, h->io, n * nrhs * 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPMC_OK;
}

// mpmc_trace_levels in three stages, so that a batch of handles can capture the
// launches of many traces in one CUDA graph: checks and every allocation; the
// kernel launches on h->stream (no allocation, no host synchronisation); the
// copy of the samples to the host and the statistics.
int trace_prepare(mpmc_ctx* h, int nsamples, int first, int* nb_out) {
    if (!h) return MPMC_EINVAL;
    if (nsamples < 1 || first < 0) return fail(h, MPMC_EINVAL, "nsamples must be >= 1 and first >= 0");
    const int L = num_levels(h);
    if (L == 0) return fail(h, MPMC_ESTATE, "no polynomial set");
    const int nb = std::min(default_nb(h), nsamples);
    if (int rc = ensure_ws(h, h->ws, h->storage, nb)) return rc;
    if (int rc = ensure_defl_work(h, nb)) return rc;
    const size_t need = (size_t)L * nsamples;
    if (h->samples_cap < need) {
        dev_free(h->samples);
        h->samples_cap = 0;
        if (int rc = dev_alloc(h, &h->samples, sizeof(double2) * need)) return rc;
        h->samples_cap = need;
    }
    if (h->polys[0].kind == MPMC_DEFLATED_COMPOSITE)
        if (int rc = ensure_projection(h)) return rc;
    *nb_out = nb;
    return MPMC_OK;
}

int trace_enqueue(mpmc_ctx* h, uint64_t seed, int nsamples, int first, int nb, int l0 = 0, int l1 = -1) {
    const int L = num_levels(h);
    if (l1 < 0) l1 = L;
    Workspace& ws = h->ws;
    for (int l = l0; l < l1; ++l) {
        const bool has_lo = l + 1 < L;
        const bool proj = h->polys[l].kind == MPMC_DEFLATED_COMPOSITE;
        const bool defl = has_lo && h->k > 0;
        for (int b0 = 0; b0 < nsamples; b0 += nb) {
            const int nvalid = std::min(nb, nsamples - b0);
            const NoiseSpec ns{seed, (uint32_t)l, (uint32_t)(first + b0)};
            cd c_hi = 0.0, c_lo = 0.0;
            if (defl || proj)
                if (int rc = deflation_dots(h, nb, ns)) return rc;
            if (proj) {
                // r = b - (A Z) D with D = H^{-1} U^H b; the sample adds b^H Z D
                launch_proj_coef(h->k, nb, h->d_pair, h->d_invd, h->d_Hinv, h->G1, h->G2, h->D, h->D32, h->xz,
                                 h->stream);
                begin_chain(h, ns, 0x7072u);
                launch_rank_update(proj_math(h), h->storage, h->g.V, nb, h->Wb, h->k, h->D, h->D32, -1.0, nullptr,
                                   ns, ws.r, h->stream, next_salt(h));
                LAUNCHED(2);
                if (int rc = chain_trace(h, ws, h->polys[l], ns, ws.r, ws.acc_hi, &c_hi)) return rc;
            } else {
                if (int rc = chain_trace(h, ws, h->polys[l], ns, nullptr, ws.acc_hi, &c_hi)) return rc;
            }
            if (has_lo)
                if (int rc = chain_trace(h, ws, h->polys[l + 1], ns, nullptr, ws.acc_lo, &c_lo)) return rc;
            if (defl) {
                launch_defl_term(h->k, nb, h->d_coef + (size_t)l * h->k, h->d_pair, h->G1, h->G2, h->dterm,
                                 h->stream);
                LAUNCHED(1);
            }
            double chi[2], clo[2];
            setc(chi, c_hi);
            setc(clo, c_lo);
            launch_finalize(ws.acc_rows, nb, nvalid, ws.acc_hi, has_lo ? ws.acc_lo : nullptr, chi, clo,
                            defl ? h->dterm : nullptr, h->samples + (size_t)l * nsamples + b0, nullptr, nullptr,
                            h->stream, proj ? h->xz : nullptr);
            LAUNCHED(1);
        }
    }
    return MPMC_OK;
}

int trace_collect(mpmc_ctx* h, int nsamples, double* mean, double* var, double* samples, int l0 = 0,
                  int l1 = -1) {
    const int L = num_levels(h);
    if (l1 < 0) l1 = L;
    const size_t need = (size_t)L * nsamples;
    std::vector<double2> hs(need);
    CK(cudaMemcpyAsync(hs.data(), h->samples, sizeof(double2) * need, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (int rc = prof_collect(h)) return rc;
    if (int rc = device_flag(h)) return rc;
    for (size_t i = (size_t)l0 * nsamples; i < (size_t)l1 * nsamples; ++i)
        if (!std::isfinite(hs[i].x) || !std::isfinite(hs[i].y)) return fail(h, MPMC_ENONFINITE, "non-finite sample");
    for (int l = l0; l < l1; ++l) {
        const double2* s = hs.data() + (size_t)l * nsamples;
        double mr = 0, mi = 0;
        for (int j = 0; j < nsamples; ++j) { mr += s[j].x; mi += s[j].y; }
        mr /= nsamples;
        mi /= nsamples;
        double v = NAN;
        if (nsamples > 1) {
            v = 0;
            for (int j = 0; j < nsamples; ++j) v += (s[j].x - mr) * (s[j].x - mr);
            v /= (nsamples - 1);
        }
        double corr[2] = {0, 0};
        if (int rc = mpmc_level_info(h, l, corr, nullptr)) return rc;
        if (mean) { mean[2 * l] = mr + corr[0]; mean[2 * l + 1] = mi + corr[1]; }
        if (var) var[l] = v;
        if (samples)
            for (int j = 0; j < nsamples; ++j) {
                samples[2 * ((size_t)l * nsamples + j)] = s[j].x;
                samples[2 * ((size_t)l * nsamples + j) + 1] = s[j].y;
            }
    }
    return MPMC_OK;
}

int mpmc_trace_levels(mpmc_handle h, uint64_t seed, int nsamples, int first, double* mean, double* var,
                      double* samples) {
    if (!h) return MPMC_EINVAL;
    int nb = 0;
    if (int rc = trace_prepare(h, nsamples, first, &nb)) return rc;
    if (int rc = trace_enqueue(h, seed, nsamples, first, nb)) return rc;
    return trace_collect(h, nsamples, mean, var, samples);
}

int mpmc_trace_level(mpmc_handle h, int level, uint64_t seed, int nsamples, int first, double* mean, double* var,
                     double* samples) {
    if (!h) return MPMC_EINVAL;
    const int L = num_levels(h);
    if (level < 0 || level >= L) return fail(h, MPMC_EINVAL, "level out of range");
    int nb = 0;
    if (int rc = trace_prepare(h, nsamples, first, &nb)) return rc;
    if (int rc = trace_enqueue(h, seed, nsamples, first, nb, level, level + 1)) return rc;
    std::vector<double> m(2 * (size_t)L), v(L);
    std::vector<double> all(samples ? 2 * (size_t)L * nsamples : 0);
    if (int rc = trace_collect(h, nsamples, m.data(), v.data(), samples ? all.data() : nullptr, level, level + 1))
        return rc;
    if (mean) { mean[0] = m[2 * level]; mean[1] = m[2 * level + 1]; }
    if (var) var[0] = v[level];
    if (samples) std::copy(all.begin() + 2 * (size_t)level * nsamples, all.begin() + 2 * (size_t)(level + 1) * nsamples,
                           samples);
    return MPMC_OK;
}

int mpmc_arnoldi(mpmc_handle h, int op_poly, const double* v0, int m, double* hbar, double* basis, int* steps) {
    if (!h) return MPMC_EINVAL;
    if (!v0 || !hbar || m < 1 || m > 4096) return fail(h, MPMC_EINVAL, "bad arnoldi arguments");
    if (op_poly >= MPMC_MAX_POLYS || (op_poly >= 0 && !h->polys[op_poly].set))
        return fail(h, MPMC_ESTATE, "operator polynomial not set");
    if (op_poly >= 0 && h->polys[op_poly].kind == MPMC_DEFLATED_COMPOSITE)
        return fail(h, MPMC_ENOTSUP, "arnoldi on a projected composite is not supported");
    const size_t n = nsites12(h);
    if (int rc = ensure_ws(h, h->ws64, ST_F64, 1)) return rc;
    double2* Vb = reinterpret_cast<double2*>(basis);
    double2* own = nullptr;
    if (!Vb) {
        if (int rc = dev_alloc(h, &own, sizeof(double2) * n * (m + 1))) return rc;
        Vb = own;
    }
    if (h->kr_m < m + 1) {
        dev_free(h->kr_part);
        dev_free(h->kr_h);
        dev_free(h->kr_nrm);
        h->kr_m = 0;
        const int np = mdot_parts(n);
        if (int rc = dev_alloc(h, &h->kr_part, sizeof(double2) * (size_t)np * (m + 1))) { dev_free(own); return rc; }
        if (int rc = dev_alloc(h, &h->kr_h, sizeof(double2) * 2 * (m + 1))) { dev_free(own); return rc; }
        if (int rc = dev_alloc(h, &h->kr_nrm, sizeof(double) * (np + 1))) { dev_free(own); return rc; }
        h->kr_m = m + 1;
    }
    int rc = MPMC_OK;
    std::fill(hbar, hbar + 2 * (size_t)(m + 1) * m, 0.0);
    Workspace& ws = h->ws64;
    double2* w = reinterpret_cast<double2*>(ws.w[2]);
    double2* tmp = reinterpret_cast<double2*>(ws.w[3]);
    double* part = reinterpret_cast<double*>(h->kr_part);
    double* nrm = h->kr_nrm;
    std::vector<double2> h1(m + 1), h2(m + 1);
    int done = 0;
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(w, v0, n * 16, cudaMemcpyHostToDevice, h->stream));
        launch_norm2(n, w, part, nrm, h->stream);
        launch_normalize(n, w, nrm, Vb, h->stream);
        LAUNCHED(3);
        for (int j = 0; j < m; ++j) {
            double2* vj = Vb + (size_t)j * n;
            if (op_poly < 0) {
                if (int e = apply_A(h, ws, vj, w)) return e;
            } else {
                if (int e = chain_apply(h, ws, h->polys[op_poly], vj, ws.r)) return e;
                if (int e = apply_A(h, ws, ws.r, w)) return e;
            }
            // two passes of classical Gram-Schmidt
            launch_mdot(n, j + 1, Vb, w, h->kr_part, h->kr_h, h->stream);
            launch_maxpy(n, j + 1, Vb, h->kr_h, w, h->stream);
            CK(cudaMemcpyAsync(h1.data(), h->kr_h, sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost, h->stream));
            launch_mdot(n, j + 1, Vb, w, h->kr_part, h->kr_h + (m + 1), h->stream);
            launch_maxpy(n, j + 1, Vb, h->kr_h + (m + 1), w, h->stream);
            CK(cudaMemcpyAsync(h2.data(), h->kr_h + (m + 1), sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost,
                               h->stream));
            launch_norm2(n, w, part, nrm, h->stream);
            LAUNCHED(8);
            double nn = 0;
            CK(cudaMemcpyAsync(&nn, nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            if (int e = prof_collect(h)) return e;
            for (int i = 0; i <= j; ++i) {
                hbar[2 * ((size_t)i * m + j)] = h1[i].x + h2[i].x;
                hbar[2 * ((size_t)i * m + j) + 1] = h1[i].y + h2[i].y;
            }
            const double beta = std::sqrt(nn);
            hbar[2 * ((size_t)(j + 1) * m + j)] = beta;
            done = j + 1;
            if (!(beta > 0) || !std::isfinite(beta)) break;
            launch_normalize(n, w, nrm, Vb + (size_t)(j + 1) * n, h->stream);
            LAUNCHED(1);
            (void)tmp;
        }
        CK(cudaStreamSynchronize(h->stream));
        return MPMC_OK;
    };
    rc = body();
    dev_free(own);
    if (steps) *steps = done;
    return rc;
}

int mpmc_combine(mpmc_handle h, const double* Vb, int m, const double* Y, int k, double* Z) {
    if (!h) return MPMC_EINVAL;
    if (!Vb || !Y || !Z || m < 1 || k < 1) return fail(h, MPMC_EINVAL, "bad combine arguments");
    const size_t n = nsites12(h);
    double2* dY = nullptr;
    if (int rc = dev_alloc(h, &dY, sizeof(double2) * (size_t)m * k)) return rc;
    int rc = cuda_check(h, cudaMemcpyAsync(dY, Y, sizeof(double2) * (size_t)m * k, cudaMemcpyHostToDevice, h->stream),
                        "copy Y");
    if (!rc) {
        launch_combine(n, m, reinterpret_cast<const double2*>(Vb), dY, k, reinterpret_cast<double2*>(Z), h->stream);
        h->launches += 1;
        rc = cuda_check(h, cudaGetLastError(), "combine");
        if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "combine");
    }
    dev_free(dY);
    return rc;
}

int mpmc_profile(mpmc_handle h, int enable) {
    if (!h) return MPMC_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    if (int rc = prof_collect(h)) return rc;
    if (enable) {
        for (int c = 0; c < 8; ++c) { h->prof_ms[c] = 0; h->prof_n[c] = 0; h->prof_b[c] = 0; }
    }
    h->prof = enable != 0;
    return MPMC_OK;
}

int mpmc_profile_read(mpmc_handle h, int cls, double* ms, long long* launches, double* bytes) {
    if (!h) return MPMC_EINVAL;
    if (cls < 0 || cls > 6) return fail(h, MPMC_EINVAL, "profile class out of range");
    CK(cudaStreamSynchronize(h->stream));
    if (int rc = prof_collect(h)) return rc;
    if (ms) *ms = h->prof_ms[cls];
    if (launches) *launches = h->prof_n[cls];
    if (bytes) *bytes = h->prof_b[cls];
    return MPMC_OK;
}

int mpmc_set_links(mpmc_handle h, const double* links) {
    if (h) ++h->gen;
    if (!h) return MPMC_EINVAL;
    if (!links) return fail(h, MPMC_EINVAL, "null links");
    const size_t nl = (size_t)h->g.V * 36;
    if (int rc = ensure_io(h, nl)) return rc;
    CK(cudaMemcpyAsync(h->io, links, nl * 16, cudaMemcpyHostToDevice, h->stream));
    launch_links(ST_F64, h->g.V, h->io, h->links64, h->stream);
    LAUNCHED(1);
    h->proj_ready = false;   // A Z changes with the links
    if (h->links32) {
        launch_links(ST_F32, h->g.V, h->io, h->links32, h->stream, h->kappa);
        launch_links_expanded(h->g.V, h->io, h->links_ex, h->stream, h->kappa);
        LAUNCHED(2);
    }
    CK(cudaStreamSynchronize(h->stream));
    return MPMC_OK;
}

int mpmc_set_launch(mpmc_handle h, int R, int bx, int sl) {
    if (h) ++h->gen;
    if (!h) return MPMC_EINVAL;
    if (R < 0 || R > 2 || bx < 0 || bx > 256 || (bx & (bx - 1)) || sl < 0 || sl > 16)
        return fail(h, MPMC_EINVAL, "launch shape out of range");
    h->tune_R = R ? R : 1;
    h->tune_bx = bx ? bx : 64;
    h->tune_sl = sl ? sl : 1;
    return MPMC_OK;
}

int mpmc_get_launch(mpmc_handle h, int* nb, int* R, int* bx, int* sl) {
    if (!h) return MPMC_EINVAL;
    if (nb) *nb = default_nb(h);
    if (R) *R = h->tune_R;
    if (bx) *bx = h->tune_bx;
    if (sl) *sl = h->tune_sl;
    return MPMC_OK;
}

int mpmc_autotune(mpmc_handle h, int max_nb, int steps) {
    if (h) ++h->gen;
    if (!h) return MPMC_EINVAL;
    if (max_nb < 1 || max_nb > MPMC_MAX_BLOCK) return fail(h, MPMC_EINVAL, "max_nb out of range");
    if (steps < 1) steps = 6;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const bool prof = h->prof;
    h->prof = false;
    const int nbs[] = {16, 32, 64, 128, 256, 512, 1024};
    const int bxs[] = {16, 32, 64};
    const int sls[] = {1, 2};
    const NoiseSpec ns{0x5eedULL, 0, 0};
    int rc = MPMC_OK;
    // time a chain of `steps` launches of one class: 0 dotted (noise-started), 1 undotted, 2 outer
    auto time_class = [&](int nb, int cls, double* per) -> int {
        if (rc) return rc;
        if ((rc = ensure_ws(h, h->ws, h->storage, nb))) return rc;
        Workspace& ws = h->ws;
        auto chain = [&]() -> int {
            for (int j = 0; j < steps; ++j) {
                if (cls < 2) {
                    StepArgs a{};
                    a.in = (cls == 0 && j == 0) ? nullptr : ws.w[j % 2 == 0 ? 1 : 0];
                    a.out = ws.w[j % 2];
                    a.dot = cls == 0;
                    setc(a.alpha, 0.5);
                    a.kappa = kap(h, h->storage);
                    setc(a.dot_w, 1.0);
                    a.acc = ws.acc_hi;
                    if (int r = step_launch(h, ws, a, ns)) return r;
                } else {
                    OuterArgs o{};
                    o.in = ws.w[0];
                    o.w = ws.w[2 + j % 2];
                    o.wout = ws.w[3 - j % 2];
                    o.y = ws.y;
                    setc(o.alpha, 0.5);
                    setc(o.beta, 0.25);
                    setc(o.gamma, 0.125);
                    o.kappa = kap(h, h->storage);
                    if (int r = outer_launch(h, ws, o, ns)) return r;
                }
            }
            return cuda_check(h, cudaGetLastError(), "autotune launch");
        };
        if ((rc = chain())) return rc;   // warm-up
        if ((rc = cuda_check(h, cudaEventRecord(e0, h->stream), "event"))) return rc;
        if ((rc = chain())) return rc;
        if ((rc = cuda_check(h, cudaEventRecord(e1, h->stream), "event"))) return rc;
        if ((rc = cuda_check(h, cudaEventSynchronize(e1), "event"))) return rc;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        h->launches += 2 * steps;
        *per = ms / ((double)steps * nb * h->g.V);
        return MPMC_OK;
    };
    const int user_sweep = h->use_sweep, user_fast = h->use_fast;
    // phase 1: block width and kernel of the dotted steps (the trace-mode chain)
    double best = INFINITY;
    int bnb = 0, bR = 1, bbx = 64, bsl = 1, bfast = 0, bsweep = 0, bts = 0, bfsl = 1;
    for (int nb : nbs) {
        if (nb > max_nb) break;
        // the six work vectors of a block must stay within ~24 GB
        if ((size_t)h->g.V * 12 * storage_bytes(h->storage) * 7 * nb > ((size_t)24 << 30)) break;
        auto consider = [&](double per) {
            if (per < best) {
                best = per; bnb = nb; bR = h->ws.cfg.R; bbx = h->tune_bx; bsl = h->tune_sl;
                bfast = h->use_fast; bfsl = h->fast_sl; bsweep = h->use_sweep; bts = h->sweep_ts;
            }
        };
        double per;
        h->use_sweep = 0;
        h->use_fast = 0;
        for (int R = 1; R <= 2 && !rc; ++R)
            for (int bx : bxs)
                for (int sl : sls) {
                    if (nb / R < bx && bx != bxs[0]) continue;
                    h->tune_R = R; h->tune_bx = bx; h->tune_sl = sl;
                    if (time_class(nb, 0, &per)) break;
                    consider(per);
                }
        if (!rc && (user_fast & 1) && fast_supported(h->storage, nb)) {
            h->use_fast = 1;
            for (int fsl : {1, 2, 4}) {
                h->fast_sl = fsl;
                if (time_class(nb, 0, &per)) break;
                consider(per);
            }
            if (!rc && (user_sweep & 1) && fsweep_supported(h->storage, h->g, nb)) {
                // t-sweep form, with links read from global memory, (bit 16) staged with the planes,
                // (bit 32) staged, one warp per site, and (bit 64) staged, two sites per warp
                for (int v : {0, 16, 32, 64}) {
                    if (v && !(user_sweep & v)) continue;
                    if (v == 32 && fsweep_variant(32, nb) != 2) continue;
                    h->use_sweep = 1 | v;
                    for (int ts = h->g.lt; ts >= 2 && !rc; ts = (ts % 2 == 0 ? ts / 2 : 1)) {
                        h->sweep_ts = ts;
                        if (time_class(nb, 0, &per)) break;
                        consider(per);
                    }
                }
            }
        } else if (!rc && (user_sweep & 8) && sweep_supported(h->storage, h->g, nb)) {
            h->use_sweep = 8;
            h->tune_R = 1; h->tune_bx = 32; h->tune_sl = 1;
            for (int ts = h->g.lt; ts >= 2 && !rc; ts = (ts % 2 == 0 ? ts / 2 : 1)) {
                h->sweep_ts = ts;
                if (time_class(nb, 0, &per)) break;
                consider(per);
            }
        }
        if (rc) break;
    }
    if (!rc && bnb == 0) rc = fail(h, MPMC_ENOMEM, "no block size fits the memory budget");
    // phase 2: at that width, the undotted and outer classes choose among the site-parallel
    // kernel, the issue-lean kernel and its t-sweep form with the parameters found above
    int fast_mask = bfast & 1, sweep_mask = bsweep & 121;
    if (!rc) {
        h->tune_R = bR; h->tune_bx = bbx; h->tune_sl = bsl;
        h->fast_sl = bfsl;
        h->sweep_ts = bts;
        for (int cls = 1; cls <= 2 && !rc; ++cls) {
            const int bit = 1 << cls;
            double bper = INFINITY;
            int bf = 0, bs = 0;
            const bool can_fast = (user_fast & bit) && fast_supported(h->storage, bnb);
            const bool can_sweep = can_fast && (user_sweep & bit) && fsweep_supported(h->storage, h->g, bnb);
            for (int c = 0; c < 3 && !rc; ++c) {
                if ((c >= 1 && !can_fast) || (c == 2 && !can_sweep)) continue;
                h->use_fast = c >= 1 ? bit : 0;
                h->use_sweep = (c == 2 ? bit | (bsweep & 112) : 0) | (bsweep & 8);
                double per;
                if (time_class(bnb, cls, &per)) break;
                if (per < bper) { bper = per; bf = c >= 1; bs = c == 2; }
            }
            if (bf) fast_mask |= bit;
            if (bs) sweep_mask |= bit;
        }
    }
    h->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        h->use_sweep = user_sweep;
        h->use_fast = user_fast;
        return rc;
    }
    h->nb_user = bnb;
    h->tune_R = bR;
    h->tune_bx = bbx;
    h->tune_sl = bsl;
    h->use_fast = fast_mask;
    h->fast_sl = bfsl;
    h->use_sweep = sweep_mask;
    h->sweep_ts = bts;
    // phase 3: with polynomials set, time one block of the handle's own multilevel trace for the
    // class assignment found above and a few alternatives, and keep the fastest
    const int L = num_levels(h);
    if (L > 0 && fast_supported(h->storage, bnb) && (user_fast & 7)) {
        std::vector<double> mean(2 * (size_t)L), var(L);
        // (fast mask, sweep mask, site-parallel shape R, bx, sl)
        struct Cand { int f, sw, R, bx, sl; };
        std::vector<Cand> cand = {{fast_mask, sweep_mask, bR, bbx, bsl}};
        const bool fsw = fsweep_supported(h->storage, h->g, bnb);
        const int shapes[][3] = {{bR, bbx, bsl}, {1, 32, 2}, {1, 64, 1}, {2, 32, 1}};
        for (const auto& sh : shapes)
            for (int fm : {0, 1, 3, 5, 7})
                for (int sm : {0, 7, 23, 39, 71}) {
                    if (sm && !fsw) continue;
                    if (fm == 7 && sh != shapes[0]) continue;   // no site-parallel step left to shape
                    // the links-staged t-sweep forms (bits 16, 32) only with the shape found in phase 1
                    if (sm > 7 && (sh != shapes[0] || !(user_sweep & sm & 112) || !(fm & 7))) continue;
                    if (sm == 39 && fsweep_variant(32, bnb) != 2) continue;
                    const int f = fm & user_fast;
                    const int sw = (sm & f & user_sweep) | (sm & user_sweep & 112) | (bsweep & 8);
                    cand.push_back({f, sw, sh[0], sh[1], sh[2]});
                }
        double tbest = INFINITY;
        Cand best_c = cand[0];
        const bool prof3 = h->prof;
        h->prof = false;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        int rc3 = MPMC_OK;
        for (size_t c = 0; c < cand.size() && !rc3; ++c) {
            h->use_fast = cand[c].f;
            h->use_sweep = cand[c].sw;
            h->tune_R = cand[c].R;
            h->tune_bx = cand[c].bx;
            h->tune_sl = cand[c].sl;
            if (c == 0) rc3 = mpmc_trace_levels(h, 0x5eedULL, bnb, 0, mean.data(), var.data(), nullptr);   // warm-up
            if (rc3) break;
            cudaEventRecord(e0, h->stream);
            rc3 = mpmc_trace_levels(h, 0x5eedULL, bnb, 0, mean.data(), var.data(), nullptr);
            cudaEventRecord(e1, h->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!rc3 && ms < tbest) { tbest = ms; best_c = cand[c]; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        h->prof = prof3;
        h->use_fast = best_c.f;
        h->use_sweep = best_c.sw;
        h->tune_R = best_c.R;
        h->tune_bx = best_c.bx;
        h->tune_sl = best_c.sl;
        if (rc3) return rc3;
    }
    return ensure_ws(h, h->ws, h->storage, bnb);
}

int mpmc_set_option(mpmc_handle h, int option, int value) {
    if (h) ++h->gen;
    if (!h) return MPMC_EINVAL;
    switch (option) {
        case MPMC_OPT_TENSOR_CORE_DEFLATION:
            h->use_tc = value != 0;
            return MPMC_OK;
        case MPMC_OPT_SWEEP_STENCIL:
            if (value < 0 || value > 127) return fail(h, MPMC_EINVAL, "sweep option is a mask in 0 .. 127");
            h->use_sweep = value;
            return MPMC_OK;
        case MPMC_OPT_SWEEP_SEGMENT:
            if (value < 0 || value > h->g.lt) return fail(h, MPMC_EINVAL, "t-segment length out of range");
            h->sweep_ts = value;
            return MPMC_OK;
        case MPMC_OPT_FAST_STENCIL:
            if (value < 0 || value > 7) return fail(h, MPMC_EINVAL, "fast-stencil option is a mask in 0 .. 7");
            h->use_fast = value;
            return MPMC_OK;
        case MPMC_OPT_FAST_SITES:
            if (value < 1 || value > 16) return fail(h, MPMC_EINVAL, "sites per thread out of range");
            h->fast_sl = value;
            return MPMC_OK;
        case MPMC_OPT_WAIT_LIMIT:
            if (value < 1 || value > 4000000) return fail(h, MPMC_EINVAL, "wait limit out of range (1 .. 4000000)");
            h->wait_limit = 1000LL * value;
            return MPMC_OK;
        case MPMC_OPT_TEST_SKIP_COPY:
            if (value < 0) return fail(h, MPMC_EINVAL, "skip-copy index must be >= 0");
            h->skip_copy = value;
            return MPMC_OK;
        case MPMC_OPT_SWEEP_ORDER:
            if (value < 0 || value > 1) return fail(h, MPMC_EINVAL, "sweep order is 0 (plain) or 1 (Morton)");
            h->sweep_order = value;
            return MPMC_OK;
        default:
            return fail(h, MPMC_EINVAL, "unknown option");
    }
}

namespace {
int cur_nb(const mpmc_ctx* h) { return h->ws.nb > 0 ? h->ws.nb : default_nb(h); }
}  // namespace

int mpmc_get_option(mpmc_handle h, int option, int* value) {
    if (!h || !value) return MPMC_EINVAL;
    switch (option) {
        case MPMC_OPT_TENSOR_CORE_DEFLATION:
            *value = (h->use_tc && h->tc_ready && h->storage != ST_F64) ? 1 : 0;
            return MPMC_OK;
        case MPMC_OPT_SWEEP_STENCIL: {
            int v = 0;
            if (fast_supported(h->storage, cur_nb(h)) && fsweep_supported(h->storage, h->g, cur_nb(h)))
                v |= h->use_sweep & h->use_fast & 7;
            if (sweep_supported(h->storage, h->g, cur_nb(h))) v |= h->use_sweep & 8;
            if (v & 7) {
                const int var = fsweep_variant(h->use_sweep, cur_nb(h));
                v |= var == 3 ? 64 : var == 2 ? 32 : var == 1 ? 16 : 0;
            }
            *value = v;
            return MPMC_OK;
        }
        case MPMC_OPT_SWEEP_SEGMENT:
            *value = ((h->use_fast & 7) && fsweep_supported(h->storage, h->g, cur_nb(h)))
                         ? fsweep_config(h->g, cur_nb(h), h->sweep_ts, fsweep_variant(h->use_sweep, cur_nb(h))).ts
                         : sweep_config(h->g, cur_nb(h), h->sweep_ts).ts;
            return MPMC_OK;
        case MPMC_OPT_FAST_STENCIL:
            *value = fast_supported(h->storage, cur_nb(h)) ? (h->use_fast & 7) : 0;
            return MPMC_OK;
        case MPMC_OPT_FAST_SITES:
            *value = h->fast_sl;
            return MPMC_OK;
        case MPMC_OPT_WAIT_LIMIT:
            *value = (int)(h->wait_limit / 1000);
            return MPMC_OK;
        case MPMC_OPT_TEST_SKIP_COPY:
            *value = h->skip_copy;
            return MPMC_OK;
        case MPMC_OPT_SWEEP_ORDER:
            *value = h->sweep_order;
            return MPMC_OK;
        default:
            return fail(h, MPMC_EINVAL, "unknown option");
    }
}

int mpmc_deflation_dots(mpmc_handle h, uint64_t seed, int level, int first, int nrhs, double* G1, double* G2) {
    if (!h) return MPMC_EINVAL;
    if (h->k == 0) return fail(h, MPMC_ESTATE, "no deflation vectors set");
    if (nrhs < 1 || nrhs > MPMC_MAX_BLOCK || level < 0 || first < 0 || !G1 || !G2)
        return fail(h, MPMC_EINVAL, "bad deflation_dots arguments");
    if (int rc = ensure_defl_work(h, nrhs)) return rc;
    const NoiseSpec ns{seed, (uint32_t)level, (uint32_t)first};
    const bool tcore = h->storage != ST_F64 && h->use_tc && h->tc_ready;
    if (tcore) {
        int tsplit, kbps;
        size_t pf;
        tc_defl_plan(h->g.V, h->k, nrhs, &tsplit, &kbps, &pf);
        if (h->tc_part_cap < pf) {
            dev_free(h->tc_part);
            h->tc_part_cap = 0;
            if (int rc = dev_alloc(h, &h->tc_part, pf * sizeof(float))) return rc;
            h->tc_part_cap = pf;
        }
        if (tc_defl_launch(h->tmap, h->g.V, h->k, nrhs, ns, h->tc_part, tsplit, kbps, h->G1, h->G2, h->d_err,
                           h->stream))
            return fail(h, MPMC_ECUDA, "tensor-core deflation kernel setup failed");
        LAUNCHED(2);
    } else {
        const int nsplit = defl_nsplit(h->g.V);
        launch_defl_dots(h->storage == ST_F64 ? ST_F64 : ST_F32, h->g, h->k, h->Z, nrhs, ns, h->defl_part, nsplit,
                         h->stream);
        launch_defl_reduce(h->k, nrhs, nsplit, h->defl_part, h->d_coef, h->d_pair, h->G1, h->G2, h->dterm, h->stream);
        LAUNCHED(3);
    }
    const size_t cnt = (size_t)h->k * nrhs;
    CK(cudaMemcpyAsync(G1, h->G1, cnt * 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(G2, h->G2, cnt * 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return device_flag(h);
}

int mpmc_set_deflation(mpmc_handle h, const double* Z, const double* lambda, const int* pair, int k) {
    if (h) ++h->gen;
    return set_deflation_impl(h, Z, lambda, pair, k, 0);
}

int mpmc_set_deflation_device(mpmc_handle h, const double* Z, const double* lambda, const int* pair, int k) {
    if (h) ++h->gen;
    return set_deflation_impl(h, Z, lambda, pair, k, 1);
}

int mpmc_vector_stats(mpmc_handle h, const double* Z, int k, double* stats) {
    if (!h) return MPMC_EINVAL;
    if (!Z || !stats || k < 1) return fail(h, MPMC_EINVAL, "bad vector_stats arguments");
    const int chunk = std::min(k, 64);
    if (int rc = ensure_ws(h, h->ws64, ST_F64, chunk)) return rc;
    const int nsplit = gram_nsplit(h->g.V);
    if (int rc = ensure_gram_part(h, (size_t)(nsplit + 1) * chunk * 2)) return rc;
    double* part = reinterpret_cast<double*>(h->gram_part);
    double* out = part + (size_t)nsplit * chunk * 4;
    Workspace& ws = h->ws64;
    std::vector<double> host((size_t)chunk * 4);
    for (int c0 = 0; c0 < k; c0 += chunk) {
        const int cnt = std::min(chunk, k - c0);
        // columns c0..c0+cnt of the vector-major input -> block layout (zero padded)
        CK(cudaMemsetAsync(ws.w[0], 0, (size_t)nsites12(h) * chunk * 16, h->stream));
        launch_vec_to_block(ST_F64, h->g.V, cnt, Z + (size_t)c0 * nsites12(h) * 2, ws.w[0], h->stream);
        if (cnt != chunk) {
            // vec_to_block wrote a block of width cnt: re-layout into width `chunk` through w[2]
            launch_import(ST_F64, h->g.V, reinterpret_cast<const double*>(ws.w[0]), cnt, 0, cnt, ws.w[2], chunk,
                          h->stream);
            CK(cudaMemcpyAsync(ws.w[0], ws.w[2], (size_t)nsites12(h) * chunk * 16, cudaMemcpyDeviceToDevice,
                               h->stream));
        }
        LAUNCHED(cnt != chunk ? 2 : 1);
        if (int rc = apply_A(h, ws, ws.w[0], ws.w[1])) return rc;
        launch_col_stats(h->g.V, chunk, reinterpret_cast<const double*>(ws.w[0]),
                         reinterpret_cast<const double*>(ws.w[1]), part, nsplit, out, h->stream);
        LAUNCHED(2);
        CK(cudaMemcpyAsync(host.data(), out, sizeof(double) * 4 * chunk, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        std::copy(host.begin(), host.begin() + 4 * cnt, stats + 4 * (size_t)c0);
    }
    return MPMC_OK;
}

int mpmc_project(mpmc_handle h, const double* B, double* R, int nrhs, int on_device) {
    if (!h) return MPMC_EINVAL;
    if (!B || !R || nrhs < 1) return fail(h, MPMC_EINVAL, "bad project arguments");
    if (h->k == 0) return fail(h, MPMC_ESTATE, "no deflation vectors set");
    const size_t n = nsites12(h);
    const int nb = std::min(default_nb(h), nrhs);
    if (int rc = ensure_ws(h, h->ws, h->storage, nb)) return rc;
    if (int rc = ensure_defl_work(h, nb)) return rc;
    if (int rc = ensure_projection(h)) return rc;
    const double* src = B;
    double* dst = R;
    if (!on_device) {
        if (int rc = ensure_io(h, n * nrhs)) return rc;
        CK(cudaMemcpyAsync(h->io, B, n * nrhs * 16, cudaMemcpyHostToDevice, h->stream));
        src = h->io;
        dst = h->io;
    }
    const int nsplit = gram_nsplit(h->g.V);
    if (int rc = ensure_gram_part(h, (size_t)nsplit * h->k * nb)) return rc;
    for (int c0 = 0; c0 < nrhs; c0 += nb) {
        const int cnt = std::min(nb, nrhs - c0);
        launch_import(h->storage, h->g.V, src, nrhs, c0, cnt, h->ws.r, nb, h->stream);
        launch_block_gram(proj_math(h), h->g.V, h->Zb, h->k, h->storage, h->ws.r, nb, 1, h->gram_part, nsplit, h->G2,
                          h->stream);
        launch_proj_coef(h->k, nb, h->d_pair, h->d_invd, h->d_Hinv, nullptr, h->G2, h->D, h->D32, nullptr, h->stream);
        launch_rank_update(proj_math(h), h->storage, h->g.V, nb, h->Wb, h->k, h->D, h->D32, -1.0, h->ws.r,
                           NoiseSpec{0, 0, 0}, h->ws.r, h->stream);
        launch_export(h->storage, h->g.V, h->ws.r, nb, dst, nrhs, c0, cnt, h->stream);
        LAUNCHED(6);
    }
    if (!on_device) CK(cudaMemcpyAsync(R, h->io, n * nrhs * 16, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPMC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches of handles
// The multilevel traces of several independent handles (different lattices,
// kappas, polynomials) run as parallel branches of one captured CUDA graph:
// each handle's launches stay on its own stream, forked from and joined to
// the batch's stream, so that small instances overlap on the GPU and a whole
// batch costs one graph launch on the host.  The graph is captured on the
// first call and replayed while the noise block (seed, count, first index)
// and every handle's state (polynomials, deflation, links, options, block,
// stream) stay the same; any change recaptures it.
struct mpmc_batch {
    std::vector<mpmc_handle> h;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    long long launches = 0;
    // stochastic rounding of BF16 chain stores: salt of the current chain (from its noise block and
    // polynomial) and the position of the next step in it, so that a call's random bits depend on
    // what it computes, not on the handle's history
    uint32_t sr_base = 0, sr_step = 0;
    uint64_t key_seed = 0;
    int key_n = -1, key_first = -1;
    std::vector<unsigned long long> key_gen;
    std::vector<int> nbs;
};

namespace {

void batch_drop_graph(mpmc_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->nodes = 0;
    b->key_n = -1;
}

}  // namespace

int mpmc_batch_create(mpmc_batch_handle* out, int n, const mpmc_handle* handles) {
    if (!out || n < 1 || !handles) return MPMC_EINVAL;
    *out = nullptr;
    // the legacy default stream (and the per-thread default stream) cannot be captured
    for (int i = 0; i < n; ++i)
        if (!handles[i] || !handles[i]->stream || handles[i]->stream == cudaStreamLegacy ||
            handles[i]->stream == cudaStreamPerThread)
            return MPMC_EINVAL;
    mpmc_batch* b = new (std::nothrow) mpmc_batch;
    if (!b) return MPMC_ENOMEM;
    b->h.assign(handles, handles + n);
    b->join.assign(n, nullptr);
    bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < n && ok; ++i) ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        mpmc_batch_destroy(b);
        return MPMC_ECUDA;
    }
    *out = b;
    return MPMC_OK;
}

int mpmc_batch_destroy(mpmc_batch_handle b) {
    if (!b) return MPMC_EINVAL;
    if (b->origin) cudaStreamSynchronize(b->origin);
    batch_drop_graph(b);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
    return MPMC_OK;
}

long long mpmc_batch_launch_count(mpmc_batch_handle b) { return b ? b->launches : -1; }

int mpmc_batch_trace_levels(mpmc_batch_handle b, uint64_t seed, int nsamples, int first, double* mean,
                            double* var) {
    if (!b || nsamples < 1 || first < 0) return MPMC_EINVAL;
    const int n = (int)b->h.size();
    b->nbs.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        mpmc_ctx* h = b->h[i];
        if (!h->stream || h->stream == cudaStreamLegacy || h->stream == cudaStreamPerThread)
            return fail(h, MPMC_EINVAL, "a batched handle needs its own stream");
        if (int rc = trace_prepare(h, nsamples, first, &b->nbs[i])) return rc;
    }
    bool same = b->exec && b->key_seed == seed && b->key_n == nsamples && b->key_first == first &&
                b->key_gen.size() == (size_t)n;
    for (int i = 0; i < n && same; ++i) same = b->key_gen[i] == b->h[i]->gen;
    if (!same) {
        batch_drop_graph(b);
        // one plain run first: lazy allocations and kernel attributes happen outside the capture
        for (int i = 0; i < n; ++i) {
            mpmc_ctx* h = b->h[i];
            const bool prof = h->prof;
            h->prof = false;
            const int rc = trace_enqueue(h, seed, nsamples, first, b->nbs[i]);
            h->prof = prof;
            if (rc) return rc;
        }
        for (int i = 0; i < n; ++i)
            if (cudaStreamSynchronize(b->h[i]->stream) != cudaSuccess) return cuda_check(b->h[i], cudaGetLastError(), "batch warm-up");
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return cuda_check(b->h[0], cudaGetLastError(), "batch capture");
        int rc = MPMC_OK;
        cudaError_t e = cudaEventRecord(b->fork, b->origin);
        for (int i = 0; i < n && !rc && e == cudaSuccess; ++i) {
            mpmc_ctx* h = b->h[i];
            e = cudaStreamWaitEvent(h->stream, b->fork, 0);
            if (e != cudaSuccess) break;
            const bool prof = h->prof;
            h->prof = false;
            const long long l0 = h->launches;
            rc = trace_enqueue(h, seed, nsamples, first, b->nbs[i]);
            h->launches = l0;   // captured, not launched: counted at replay
            h->prof = prof;
            if (rc) break;
            e = cudaEventRecord(b->join[i], h->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
        }
        const cudaError_t e2 = cudaStreamEndCapture(b->origin, &graph);
        if (rc || e != cudaSuccess || e2 != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            (void)cudaGetLastError();
            return rc ? rc : fail(b->h[0], MPMC_ECUDA, "batch graph capture failed");
        }
        if (cudaGraphGetNodes(graph, nullptr, &b->nodes) != cudaSuccess ||
            cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            (void)cudaGetLastError();
            b->exec = nullptr;
            return fail(b->h[0], MPMC_ECUDA, "batch graph instantiation failed");
        }
        cudaGraphDestroy(graph);
        b->key_seed = seed;
        b->key_n = nsamples;
        b->key_first = first;
        b->key_gen.resize(n);
        for (int i = 0; i < n; ++i) b->key_gen[i] = b->h[i]->gen;
    }
    if (cudaGraphLaunch(b->exec, b->origin) != cudaSuccess || cudaStreamSynchronize(b->origin) != cudaSuccess)
        return cuda_check(b->h[0], cudaGetLastError(), "batch graph launch");
    b->launches += (long long)b->nodes;
    for (int i = 0; i < n; ++i) {
        double* m = mean ? mean + 2 * (size_t)i * MPMC_MAX_POLYS : nullptr;
        double* v = var ? var + (size_t)i * MPMC_MAX_POLYS : nullptr;
        if (int rc = trace_collect(b->h[i], nsamples, m, v, nullptr)) return rc;
    }
    return MPMC_OK;
}
