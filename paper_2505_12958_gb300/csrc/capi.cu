// capi.cu -- the C ABI declared in include/ap.h: context set-up, the per-step pipeline,
// state transfer and timing.  The step pipeline is launched on one stream with no host
// synchronisation: the neighbour rebuild decision, the ACE atom count and all error
// conditions live in device memory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "ap_internal.h"

struct ap_ctx {
    ap::Ctx c;
    // the fixed-size device buffers of the context, carved from one allocation
    char* arena = nullptr;
    size_t arena_bytes = 0;
    // the fresh energies of the last force evaluation include the per-atom virial
    bool energy_virial = false;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_ev;
    // captured MD steps (kick-drift, force evaluation, kick), replayed by ap_step: one step,
    // and kStepBlock steps in one graph for long runs (one launch instead of kStepBlock)
    cudaGraphExec_t step_exec = nullptr;
    cudaGraphExec_t block_exec = nullptr;
    cudaStream_t step_stream = nullptr;
    double step_dt = 0.0;
    long long step_kernels = 0;
    long long step_gen = -1;
    // with only the ACE contraction timed: one step graph whose two event-record nodes
    // around the contraction get a fresh event pair before every replay (ev_mark are the
    // events recorded during capture, ev_node the nodes; the graph keeps the nodes valid)
    cudaGraph_t timed_graph = nullptr;
    cudaGraphExec_t timed_exec = nullptr;
    cudaGraphNode_t ev_node[2] = {nullptr, nullptr};
    cudaEvent_t ev_mark[2] = {nullptr, nullptr};
    long long timed_kernels = 0;
    long long timed_count = 0;                           // steps replayed in profiling mode 3
    // ap_compute_forces_host's kernels as one graph between its plain copies, captured per
    // (stream, buffer layout, mode: bit 0 positions given, bit 1 energy asked)
    cudaGraphExec_t host_exec = nullptr;
    cudaStream_t host_stream = nullptr;
    long long host_gen = -1;
    int host_mode = -1;
    long long host_kernels = 0;
    cudaError_t cap_err = cudaSuccess;                  // the first error inside a capture
    // the EAM passes run on a branch of their own (side), forked after the list build and
    // joined before the blend, beside the ACE basis, contraction and force kernels
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // the contraction is done: with the energies of a host-buffer evaluation, the energy blend
    // and its reduction run on the branch after it, beside the ACE force kernel
    cudaEvent_t ace_ev = nullptr;
    const char* cap_where = "";                          // the capture call that failed
};

namespace {

thread_local std::string g_init_err;
bool injected_alloc_failure();

}  // namespace

namespace ap {
// the text ap_last_error(NULL) returns on this thread: the last failed ap_init or
// ap_ace_forces_noalloc
void set_global_error(const std::string& m) { g_init_err = m; }

const AceTc* shared_ace_tables(const AceTc& host, int dev, std::string& err) {
    struct Entry { int dev; std::unique_ptr<AceTc> host; AceTc* d; };
    static std::mutex mu;
    static std::vector<Entry> cache;
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& e : cache)
        if (e.dev == dev && std::memcmp(e.host.get(), &host, sizeof(AceTc)) == 0) return e.d;
    std::unique_ptr<AceTc> copy(new (std::nothrow) AceTc(host));
    AceTc* d = nullptr;
    if (!copy || injected_alloc_failure() || cudaMalloc((void**)&d, sizeof(AceTc)) != cudaSuccess) {
        cudaGetLastError();
        err = "ACE table allocation failed";
        return nullptr;
    }
    if (cudaMemcpy(d, &host, sizeof(AceTc), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        err = "ACE table upload failed";
        return nullptr;
    }
    cache.push_back({dev, std::move(copy), d});
    return d;
}

void fill_ctx_dev(const Ctx& c, CtxDev& d) {
    std::memset(&d, 0, sizeof(d));
    d.n = c.n;
    d.ncode = c.grid.ncode;
    d.cap = c.cap;
    d.load_cap = c.load_cap;
    d.mass = c.mass;
    const double lim = 0.5 * c.skin;
    d.lim2 = lim * lim;
    d.ace_c1_0 = c.ace_c1_0;
    d.grid = c.grid;
    d.dyn = c.dyn;
    d.x = c.x; d.v = c.v; d.xb = c.xb; d.f = c.f; d.pos4 = c.pos4;
    d.uxi = c.uxi; d.w = c.w; d.e_ace = c.e_ace; d.ace_A = c.ace_A; d.ace_dA = c.ace_dA; d.vir_ace = c.vir_ace;
    d.e_emb = c.e_emb; d.e_eam = c.e_eam; d.w_fixed = c.w_fixed; d.d_time = c.d_time;
    d.acc = c.acc; d.fixed = c.fixed;
    d.cell = c.cell; d.cell_count = c.cell_count; d.cell_start = c.cell_start; d.cell_atoms = c.cell_atoms;
    d.nbr = c.nbr; d.nbr_row = c.nbr_row; d.nnbr = c.nnbr; d.ace_list = c.ace_list; d.flags = c.flags;
    d.d_step = c.d_step; d.load_ring = c.load_ring; d.load_ring_t = c.load_ring_t;
    d.eam = c.eam_d; d.ace = c.ace_tc_d; d.D = c.D;
}
}  // namespace ap

namespace {

ap_status set_err(ap::Ctx& c, ap_status s, const std::string& m) {
    c.err = m;
    return s;
}

// pending injected allocation failures (ap_inject_alloc_failures)
std::atomic<int> g_fail_allocs{0};

bool injected_alloc_failure() {
    int v = g_fail_allocs.load();
    while (v > 0)
        if (g_fail_allocs.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

ap_status cuda_check(ap::Ctx& c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return AP_OK;
    c.err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? AP_ERR_OOM : AP_ERR_CUDA;
}

cudaStream_t pick(ap_ctx* x, void* s) { return s ? (cudaStream_t)s : x->c.stream; }

cudaEvent_t get_event(ap_ctx* x) {
    if (!x->free_ev.empty()) { cudaEvent_t e = x->free_ev.back(); x->free_ev.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// fold the completed stage events at the front of the pending list into the totals and
// recycle them (no waiting), so that long profiled runs create no new events
void drain_ready(ap_ctx* x) {
    ap::Ctx& c = x->c;
    size_t k = 0;
    for (; k < x->pending.size(); ++k) {
        auto& p = x->pending[k];
        if (cudaEventQuery(p.b) != cudaSuccess) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) break;
        c.stage_ms[p.stage] += ms;
        c.stage_n[p.stage] += 1;
        x->free_ev.push_back(p.a);
        x->free_ev.push_back(p.b);
    }
    x->pending.erase(x->pending.begin(), x->pending.begin() + k);
}

// run one stage; with profiling on, bracket it with events on the same stream
template <class F>
void stage(ap_ctx* x, int st, cudaStream_t s, F&& launch) {
    ap::Ctx& c = x->c;
    if (!c.prof || (c.prof >= 2 && st != AP_STAGE_ACE)) { c.launches += launch(); return; }
    if (x->pending.size() >= 64) drain_ready(x);
    cudaEvent_t a = get_event(x), b = get_event(x);
    cudaEventRecord(a, s);
    c.launches += launch();
    cudaEventRecord(b, s);
    x->pending.push_back({st, a, b});
}

constexpr int kStepBlock = 8;

void drop_step_graph(ap_ctx* x) {
    for (cudaGraphExec_t* g : {&x->step_exec, &x->block_exec, &x->timed_exec, &x->host_exec}) {
        if (*g) cudaGraphExecDestroy(*g);
        *g = nullptr;
    }
    if (x->timed_graph) cudaGraphDestroy(x->timed_graph);
    x->timed_graph = nullptr;
    x->ev_node[0] = x->ev_node[1] = nullptr;
}

// Capture body() on s as one graph and instantiate it.  kernels = launches per replay;
// keep: the graph is handed back instead of destroyed.  Stage timing is off while capturing.
template <class F>
cudaError_t capture_graph(ap_ctx* xc, cudaStream_t s, cudaGraphExec_t* out, long long* kernels, F&& body,
                          cudaGraph_t* keep = nullptr) {
    ap::Ctx& c = xc->c;
    cudaGraph_t g = nullptr;
    xc->cap_err = cudaSuccess;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    xc->cap_where = "";
    const int prof = c.prof;
    c.prof = 0;
    const long long before = c.launches;
    body();
    *kernels = c.launches - before;
    c.launches = before;
    c.prof = prof;
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess && e2 != cudaSuccess) { e = e2; xc->cap_where = "end capture"; }
    if (e == cudaSuccess) e = xc->cap_err;
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(out, g, 0);
        if (e != cudaSuccess) xc->cap_where = "instantiate";
    }
    if (e != cudaSuccess) *out = nullptr;
    if (keep && e == cudaSuccess) *keep = g;
    else if (g) cudaGraphDestroy(g);
    return e;
}

ap_status graph_error(ap_ctx* xc, cudaError_t e) {
    const std::string what = std::string("graph capture (") + xc->cap_where + ")";
    return cuda_check(xc->c, e, what.c_str());
}

bool capturable(cudaStream_t s) {
    return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

void drain_events(ap_ctx* x) {
    ap::Ctx& c = x->c;
    for (auto& p : x->pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        c.stage_ms[p.stage] += ms;
        c.stage_n[p.stage] += 1;
        x->free_ev.push_back(p.a);
        x->free_ev.push_back(p.b);
    }
    x->pending.clear();
}

void inv3(const double* M, double* R) {
    double a = M[0], b = M[1], cc = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], i = M[8];
    double det = a * (e * i - f * h) - b * (d * i - f * g) + cc * (d * h - e * g);
    R[0] = (e * i - f * h) / det; R[1] = (cc * h - b * i) / det; R[2] = (b * f - cc * e) / det;
    R[3] = (f * g - d * i) / det; R[4] = (a * i - cc * g) / det; R[5] = (cc * d - a * f) / det;
    R[6] = (d * h - e * g) / det; R[7] = (b * g - a * h) / det; R[8] = (a * e - b * d) / det;
}

void cross(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1]; c[1] = a[2] * b[0] - a[0] * b[2]; c[2] = a[0] * b[1] - a[1] * b[0];
}

ap_status setup_grid(ap::Ctx& c, const ap_box& box, std::vector<float4>& D, std::vector<float4>& Dlo) {
    ap::GridDev& g = c.grid;
    std::memcpy(g.h, box.h, sizeof(g.h));
    std::memcpy(g.origin, box.origin, sizeof(g.origin));
    double V, cr[3];
    cross(g.h + 3, g.h + 6, cr);
    V = g.h[0] * cr[0] + g.h[1] * cr[1] + g.h[2] * cr[2];
    if (!(std::fabs(V) > 1e-9)) return set_err(c, AP_ERR_ARG, "box edge vectors are degenerate");
    inv3(g.h, g.hinv);
    double pw[3];
    for (int d = 0; d < 3; ++d) {
        const double* a = g.h + 3 * ((d + 1) % 3);
        const double* b = g.h + 3 * ((d + 2) % 3);
        cross(a, b, cr);
        pw[d] = std::fabs(V) / std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    }
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        g.periodic[d] = box.periodic[d] ? 1 : 0;
        int n = (int)std::floor(pw[d] / c.rc_list);
        n = std::max(1, std::min(n, 1024));
        g.nc[d] = n;
        int S = 1;
        if (g.periodic[d]) S = std::max(1, (int)std::ceil(c.rc_list * n / pw[d] - 1e-12));
        if (S > 2) return set_err(c, AP_ERR_ARG, "box thinner than half the neighbour-list cutoff");
        g.S[d] = S;
        ncell *= n;
        for (int q = 0; q < 3; ++q) g.cellvec[3 * d + q] = g.h[3 * d + q] / n;
        g.cw[d] = pw[d] / n;
    }
    if (ncell > (1ll << 26)) return set_err(c, AP_ERR_ARG, "cell grid too large");
    g.ortho = (g.h[1] == 0.0 && g.h[2] == 0.0 && g.h[3] == 0.0 && g.h[5] == 0.0 && g.h[6] == 0.0 && g.h[7] == 0.0) ? 1 : 0;
    for (int d = 0; d < 3; ++d) {
        g.L[d] = g.h[4 * d];
        g.Linv[d] = 1.0 / g.h[4 * d];
        g.Lf[d] = (float)g.L[d];
        g.Linvf[d] = (float)g.Linv[d];
    }
    g.ncell = (int)ncell;
    g.ncode = (2 * g.S[0] + 1) * (2 * g.S[1] + 1) * (2 * g.S[2] + 1);
    g.rlist2 = (float)(c.rc_list * c.rc_list);
    D.resize(g.ncode);
    Dlo.resize(g.ncode);
    const int w1 = 2 * g.S[1] + 1, w2 = 2 * g.S[2] + 1;
    for (int code = 0; code < g.ncode; ++code) {
        int o[3] = {code / (w1 * w2) - g.S[0], (code / w2) % w1 - g.S[1], code % w2 - g.S[2]};
        double v[3];
        for (int q = 0; q < 3; ++q) v[q] = o[0] * g.cellvec[q] + o[1] * g.cellvec[3 + q] + o[2] * g.cellvec[6 + q];
        D[code] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
        Dlo[code] = make_float4((float)(v[0] - (float)v[0]), (float)(v[1] - (float)v[1]), (float)(v[2] - (float)v[2]), 0.f);
    }
    return AP_OK;
}

// Context memory comes from the device's stream-ordered pool on the context's stream, so
// creating and destroying contexts (e.g. requests of a serving loop) never synchronises
// the whole device; freed blocks stay cached in the pool up to a release threshold.
void pool_setup(int dev) {
    static int done = -1;
    if (done == dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = 8ull << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done = dev;
}

template <class T>
ap_status dalloc(ap::Ctx& c, T** p, size_t count) {
    if (count == 0) count = 1;
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cuda_check(c, cudaErrorMemoryAllocation, "cudaMallocAsync (injected failure)");
    }
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), c.stream);
    if (e != cudaSuccess) { *p = nullptr; return cuda_check(c, e, "cudaMallocAsync"); }
    c.dev_bytes += count * sizeof(T);
    return AP_OK;
}

// Pinned host slots for each context's flag and total read-backs.  cudaFreeHost waits for
// the whole device, which would stall every other context's stream whenever one context
// is destroyed, so slots are recycled for the lifetime of the process instead.
constexpr size_t kPinnedSlot = 256;                     // 16 doubles of totals + flags
static_assert(16 * sizeof(double) + ap::kFlagCount * sizeof(int) <= kPinnedSlot, "pinned slot");
std::mutex g_pinned_mu;
std::vector<char*> g_pinned_free;

char* pinned_take() {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (g_pinned_free.empty()) {
        char* block = nullptr;
        const int per = 256;
        if (cudaMallocHost((void**)&block, kPinnedSlot * per) != cudaSuccess) return nullptr;
        for (int k = per - 1; k >= 0; --k) g_pinned_free.push_back(block + kPinnedSlot * k);
    }
    char* p = g_pinned_free.back();
    g_pinned_free.pop_back();
    return p;
}

void pinned_give(char* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned_free.push_back(p);
}

void free_all(ap_ctx* xc) {
    ap::Ctx& c = xc->c;
    void* ps[] = {c.eam_d, c.D, c.Dlo, c.pos_lo, c.ace_A, c.ace_dA, c.x, c.v, c.xb, c.f, c.pos4, c.uxi, c.w, c.e_emb, c.e_eam, c.e_ace,
                  c.vir_eam, c.vir_ace, c.acc, c.fixed, c.w_fixed, c.cell, c.cell_count, c.cell_start,
                  c.cell_atoms, c.nbr, c.nbr_tmp, c.nbr_row, c.nnbr, c.ace_list, c.flags, c.d_time, c.partials, c.totals, c.e_atom,
                  c.pos_stage, c.f_stage, c.csp_sum, c.csp_under, c.csp_w0, c.csp_wnew, c.csp_seeds, c.csp_nseed,
                  c.thermo_group, c.nh_state, c.nh_partials, c.d_step, c.com, c.load_ring, c.load_ring_t};
    for (void* p : ps) {
        const bool carved = xc->arena && (char*)p >= xc->arena && (char*)p < xc->arena + xc->arena_bytes;
        if (p && !carved) cudaFreeAsync(p, c.stream);
    }
    if (xc->arena) cudaFreeAsync(xc->arena, c.stream);
    xc->arena = nullptr;
    xc->arena_bytes = 0;
    cudaStreamSynchronize(c.stream);
    if (xc->side) cudaStreamSynchronize(xc->side);
    for (cudaEvent_t* e : {&xc->fork_ev, &xc->join_ev, &xc->ace_ev}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    if (xc->side) cudaStreamDestroy(xc->side);
    xc->side = nullptr;
    pinned_give((char*)c.h_totals);
    c.h_totals = nullptr;
    c.h_flags = nullptr;
    c.dev_bytes = 0;
    delete c.ace_h;
}

// Fixed-size buffers of a context: the sizes are gathered first, then one stream-ordered
// allocation is carved into 256-byte aligned pieces (an allocation call costs ~10 us, and a
// context has some 30 such buffers).
struct ArenaPlan {
    struct Item { void** p; size_t bytes; };
    std::vector<Item> items;
    template <class T>
    void add(T** p, size_t count) { items.push_back({(void**)p, (count ? count : 1) * sizeof(T)}); }
};

ap_status arena_commit(ap_ctx* xc, const ArenaPlan& plan) {
    ap::Ctx& c = xc->c;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t total = 0;
    for (const auto& it : plan.items) total += up(it.bytes);
    cudaError_t e = injected_alloc_failure() ? cudaErrorMemoryAllocation
                                             : cudaMallocAsync((void**)&xc->arena, total, c.stream);
    if (e != cudaSuccess) { xc->arena = nullptr; return cuda_check(c, e, "cudaMallocAsync"); }
    xc->arena_bytes = total;
    size_t off = 0;
    for (const auto& it : plan.items) {
        *it.p = xc->arena + off;
        off += up(it.bytes);
    }
    c.dev_bytes += total;
    return AP_OK;
}

void to_soa(const double* aos, int n, double* soa) {
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) soa[(size_t)k * n + i] = aos[3 * (size_t)i + k];
}

void to_soa(const double* aos, int n, std::vector<double>& soa) {
    soa.resize(3 * (size_t)n);
    to_soa(aos, n, soa.data());
}

// Pinned staging blocks for the uploads of ap_init.  A copy from pageable memory passes
// through the driver's own staging buffers and can hold the calling thread for milliseconds
// while transfers of other streams occupy them; a copy from pinned memory is queued and
// returns at once.  A block is used by one context's uploads and recycled once the event
// recorded after them has completed; blocks are never freed (like the pinned slots above).
struct Staging {
    char* p = nullptr;
    size_t bytes = 0;
    int dev = -1;
    cudaEvent_t ev = nullptr;
};
std::mutex g_stage_mu;
std::vector<Staging> g_stage_free, g_stage_busy;

bool staging_take(size_t bytes, int dev, Staging& out) {
    std::lock_guard<std::mutex> lk(g_stage_mu);
    for (size_t k = 0; k < g_stage_busy.size();) {
        if (cudaEventQuery(g_stage_busy[k].ev) == cudaSuccess) {
            g_stage_free.push_back(g_stage_busy[k]);
            g_stage_busy[k] = g_stage_busy.back();
            g_stage_busy.pop_back();
        } else {
            ++k;
        }
    }
    int best = -1;
    for (int k = 0; k < (int)g_stage_free.size(); ++k)
        if (g_stage_free[k].dev == dev && g_stage_free[k].bytes >= bytes &&
            (best < 0 || g_stage_free[k].bytes < g_stage_free[best].bytes))
            best = k;
    if (best >= 0) {
        out = g_stage_free[best];
        g_stage_free[best] = g_stage_free.back();
        g_stage_free.pop_back();
        return true;
    }
    Staging b;
    b.bytes = (size_t)1 << 20;
    while (b.bytes < bytes) b.bytes <<= 1;
    b.dev = dev;
    if (cudaMallocHost((void**)&b.p, b.bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(b.p);
        return false;
    }
    out = b;
    return true;
}

// the block's copies are queued on s: it returns to the pool when they have completed
void staging_give(const Staging& b, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (cudaEventRecord(b.ev, s) == cudaSuccess) {
        g_stage_busy.push_back(b);
    } else {
        cudaGetLastError();
        cudaStreamSynchronize(s);
        g_stage_free.push_back(b);
    }
}

// one AP force evaluation of the current positions (stages a1-a7), in two parts around the
// ACE contraction.  after_drift: the kick-drift kernel of this step already took the
// neighbour-list displacement test (positions change only there between evaluations of a
// step loop), so the separate check is left out.  kick_dt > 0: the blend kernel also
// applies the step's second half kick.
// eam_energy: the caller will ask for the total energy; the compensated EAM energies are then
// formed on the EAM branch, beside the ACE kernels (they write their own buffer, so the force
// pass's results do not change), and only the energy blend follows the force blend
void run_forces_pre(ap_ctx* xc, cudaStream_t s, bool after_drift, bool eam_energy = false) {
    ap::Ctx& c = xc->c;
    stage(xc, AP_STAGE_NEIGHBOR, s, [&] { return (after_drift ? 0 : ap::launch_check(c, s)) + ap::launch_rebuild(c, s); });
    stage(xc, AP_STAGE_PREPARE, s, [&] { return ap::launch_prepare(c, s); });
    stage(xc, AP_STAGE_NEIGHBOR, s, [&] { return ap::launch_build(c, s, 0); });
    if (c.prof == 1) {
        // every stage timed: the EAM passes stay on s, inside their own events
        stage(xc, AP_STAGE_EAM_DENSITY, s, [&] { return ap::launch_eam_density(c, s); });
        stage(xc, AP_STAGE_EAM_FORCE, s, [&] { return ap::launch_eam_force(c, s); });
    } else {
        // the EAM branch: it writes only its own buffers (f, e_eam, uxi, e_emb), and the
        // ACE kernels on s read none of them
        cudaEventRecord(xc->fork_ev, s);
        cudaStreamWaitEvent(xc->side, xc->fork_ev, 0);
        // with eam_energy the density pass also forms the compensated EAM energies (the bits
        // of the on-request energy pass without the virial)
        c.launches += eam_energy ? ap::launch_eam_density_energy(c, xc->side) : ap::launch_eam_density(c, xc->side);
        c.launches += ap::launch_eam_force(c, xc->side);
        if (!eam_energy) cudaEventRecord(xc->join_ev, xc->side);      // else after the energy blend
    }
    stage(xc, AP_STAGE_ACE_BASIS, s, [&] { return ap::launch_ace_basis(c, s); });
}

void run_forces_post(ap_ctx* xc, cudaStream_t s, float* out_aos, double kick_dt, bool in_step) {
    ap::Ctx& c = xc->c;
    stage(xc, AP_STAGE_ACE_FORCE, s, [&] { return ap::launch_ace_force(c, s); });
    if (c.prof != 1) cudaStreamWaitEvent(s, xc->join_ev, 0);      // join the EAM branch
    stage(xc, AP_STAGE_BLEND, s, [&] { return ap::launch_blend(c, s, out_aos, kick_dt, in_step); });
    c.forces_valid = true;
    c.energy_fresh = false;
}

void run_forces(ap_ctx* xc, cudaStream_t s, float* out_aos, bool after_drift = false, double kick_dt = 0.0,
                bool eam_energy = false) {
    run_forces_pre(xc, s, after_drift, eam_energy);
    stage(xc, AP_STAGE_ACE, s, [&] { return ap::launch_ace(xc->c, s); });
    if (eam_energy && xc->c.prof != 1) {
        // the energy blend reads E_i^ACE of the contraction and the branch's EAM energies, not
        // the forces: it and the total's reduction run on the branch beside the ACE force kernel
        cudaEventRecord(xc->ace_ev, s);
        cudaStreamWaitEvent(xc->side, xc->ace_ev, 0);
        xc->c.launches += ap::launch_energy_blend(xc->c, xc->side, false) + ap::launch_reduce(xc->c, xc->side, 0);
        cudaEventRecord(xc->join_ev, xc->side);
    }
    run_forces_post(xc, s, out_aos, kick_dt, after_drift);
}

// accurate energies of the last force evaluation, once
// (totals and per-atom energies; the per-atom virial only when asked for)
void ensure_energy(ap_ctx* xc, cudaStream_t s, bool virial = true) {
    ap::Ctx& c = xc->c;
    if (c.energy_fresh && (xc->energy_virial || !virial)) return;
    c.launches += ap::launch_energy(c, s, virial);
    c.energy_fresh = true;
    xc->energy_virial = virial;
}

ap_status read_flags(ap::Ctx& c, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(c.h_flags, c.flags, sizeof(int) * ap::kFlagCount, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(c, e, "synchronise");
    int err = c.h_flags[ap::kFlagErr];
    if (err & ap::kErrAceCapacity) {
        // checked first: the skipped atoms' ACE terms are not evaluated, so a domain error
        // that comes with it may be a consequence
        c.forces_valid = false;
        return set_err(c, AP_ERR_LIMIT, "more than " + std::to_string(ap::kAceNbrCap) +
                                            " neighbours within the ACE cutoff at atom " +
                                            std::to_string(c.h_flags[ap::kFlagBad]));
    }
    if (err & ap::kErrDomain)
        return set_err(c, AP_ERR_DOMAIN, "domain error (phi2 <= 1e-3, rho < 0 or non-finite) at atom " + std::to_string(c.h_flags[ap::kFlagBad]));
    if (err & ap::kErrCapacity) {
        // grow the list capacity; the next evaluation rebuilds
        int need = c.h_flags[ap::kFlagMaxNbr];
        std::string m = "neighbour capacity exceeded (" + std::to_string(need) + " > " + std::to_string(c.cap) + ")";
        ap_status grown = AP_ERR_CAPACITY;
        {
            int cap = ((int)(need * 1.25) + 8 + 3) & ~3;
            int *nb = nullptr, *nt = nullptr, *nr = nullptr;
            cudaError_t ea = injected_alloc_failure() ? cudaErrorMemoryAllocation
                                                      : cudaMallocAsync((void**)&nb, (size_t)cap * c.n * sizeof(int), c.stream);
            if (ea == cudaSuccess) {
                ea = cudaMallocAsync((void**)&nt, (size_t)cap * c.n * sizeof(int), c.stream);
                if (ea != cudaSuccess) cudaFreeAsync(nb, c.stream);
            }
            if (ea == cudaSuccess) {
                ea = cudaMallocAsync((void**)&nr, (size_t)cap * c.n * sizeof(int), c.stream);
                if (ea != cudaSuccess) {
                    cudaFreeAsync(nb, c.stream);
                    cudaFreeAsync(nt, c.stream);
                }
            }
            if (ea == cudaSuccess) {
                cudaFreeAsync(c.nbr, c.stream);
                cudaFreeAsync(c.nbr_tmp, c.stream);
                cudaFreeAsync(c.nbr_row, c.stream);
                c.dev_bytes += 3 * ((size_t)cap - (size_t)c.cap) * c.n * sizeof(int);
                c.nbr = nb;
                c.nbr_tmp = nt;
                c.nbr_row = nr;
                c.cap = cap;
                c.layout_gen += 1;
            } else {
                cudaGetLastError();
                grown = AP_ERR_OOM;
                m += "; growing the list failed (out of device memory)";
            }
        }
        int zero[2] = {1, 0};
        cudaMemcpyAsync(&c.flags[ap::kFlagRebuild], &zero[0], sizeof(int), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(&c.flags[ap::kFlagErr], &zero[1], sizeof(int), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        c.forces_valid = false;
        return set_err(c, grown, m);
    }
    return AP_OK;
}

}  // namespace

extern "C" {

int ap_version(void) { return AP_API_VERSION; }

// neighbour slots per atom for the list sphere of radius rl at 0.1 atoms / A^3 (denser than
// any metal here), with the 25 % margin and the rounding of the counted capacity
static int list_capacity_bound(double rl) {
    const double need = 4.18879 * rl * rl * rl * 0.1;
    return ((int)(need * 1.25) + 8 + 3) & ~3;
}

size_t ap_footprint_bytes(const ap_potential* pot, int n_atoms, double ace_fraction) {
    (void)ace_fraction;   // the ACE arrays are sized for every atom (the region moves)
    double rl = 6.5;
    if (pot) {
        double rc = 0.0;
        for (int k = 0; k < pot->eam_n_phi && k < 32; ++k) rc = std::max(rc, pot->eam_phi_d[k]);
        for (int k = 0; k < pot->eam_n_rho && k < 16; ++k) rc = std::max(rc, pot->eam_rho_d[k]);
        rc = std::max(rc, pot->ace_rc);
        rl = rc + (pot->skin > 0 ? pot->skin : 1.0);
    }
    // the neighbour capacity of bound sizing, which the counted capacity stays below for
    // structures of metallic density
    const size_t cap = (size_t)list_capacity_bound(rl) + 4;
    // per-atom arrays allocated by ap_init (and the host-transfer staging buffers)
    const size_t per_atom = 16 + 3 * 8 * 3 + 3 * 4 + 16 + 4 + 4 + 8 + 8 + 8 + 4 +
                            2 * sizeof(float) * ap::kNLM * ap::kNmax + 2 * 6 * 4 + 3 * 8 + 1 + 8 +
                            4 + 4 + 4 + 4 + 8 + 3 * 8 + 3 * 4 + 3 * cap * 4;   // the list, its row copy, the build's scratch
    const size_t cells = 2 * sizeof(int) * ((size_t)n_atoms + 1);   // cell count/start (<= 1 per atom)
    const size_t nred = (size_t)(n_atoms + ap::kRedBlock - 1) / ap::kRedBlock + 1;
    return (size_t)n_atoms * per_atom + cells + nred * 10 * 8 + 2 * 125 * 16 + sizeof(ap::AceTc) + 512 +
           sizeof(ap::EamDev) + (1u << 16);
}

size_t ap_memory_bytes(const ap_ctx* xc) { return xc ? xc->c.dev_bytes : 0; }

ap_status ap_init(const ap_potential* pot, const ap_box* box, const ap_region* region, const ap_indenter* ind,
                  int n, const double* pos, const double* vel, const unsigned char* fixed, void* stream,
                  ap_ctx** out) {
    if (!out) return AP_ERR_ARG;
    *out = nullptr;
    if (!pot || !box || !pos || n < 1 || n > ap::kMaxAtoms) { g_init_err = "ap_init: missing argument or bad atom count"; return AP_ERR_ARG; }
    if (!(pot->mass_amu > 0.0) || !(pot->skin >= 0.0)) { g_init_err = "ap_init: mass must be > 0 and skin >= 0"; return AP_ERR_ARG; }
    if (pot->ace_precision < AP_ACE_FP32 || pot->ace_precision > AP_ACE_FP64) { g_init_err = "ap_init: unknown ace_precision"; return AP_ERR_ARG; }
    if (pot->list_sizing != AP_LIST_COUNTED && pot->list_sizing != AP_LIST_BOUND) { g_init_err = "ap_init: unknown list_sizing"; return AP_ERR_ARG; }
    ap_ctx* xc = new (std::nothrow) ap_ctx();
    if (!xc) return AP_ERR_OOM;
    ap::Ctx& c = xc->c;
    c.n = n;
    c.mass = pot->mass_amu;
    c.skin = pot->skin;
    c.ace_prec = pot->ace_precision;
    c.stream = (cudaStream_t)stream;
    ap_status st = AP_OK;
    auto fail = [&](ap_status s2) {
        g_init_err = c.err;
        free_all(xc);
        delete xc;
        return s2;
    };
    if (cudaGetDevice(&c.dev) != cudaSuccess) { c.err = "no CUDA device"; return fail(AP_ERR_CUDA); }
    pool_setup(c.dev);
    if (cudaStreamCreateWithFlags(&xc->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&xc->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&xc->join_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&xc->ace_ev, cudaEventDisableTiming) != cudaSuccess) {
        c.err = "stream or event creation failed";
        return fail(AP_ERR_CUDA);
    }
    std::string err;
    if (ap::build_eam_tables(*pot, c.eam_h, err)) { c.err = err; return fail(AP_ERR_ARG); }
    c.ace_h = new (std::nothrow) ap::AceDev();
    if (!c.ace_h) { c.err = "host allocation"; return fail(AP_ERR_OOM); }
    if (ap::build_ace_tables(*pot, *c.ace_h, err)) { c.err = err; return fail(AP_ERR_ARG); }
    c.ace_c1_0 = pot->ace_c1_0;
    {
        static std::mutex mu;
        static std::vector<int> done;
        std::lock_guard<std::mutex> lk(mu);
        if (std::find(done.begin(), done.end(), c.dev) == done.end()) {
            std::vector<float> g(ap::kNG);
            if (ap::gaunt_values(g.data(), err)) { c.err = err; return fail(AP_ERR_ARG); }
            ap::upload_gaunt(g.data());
            done.push_back(c.dev);
        }
    }
    c.rc_eam = c.eam_h.rc;
    c.rc_ace = pot->ace_rc;
    c.rc_list = std::max(c.rc_eam, c.rc_ace) + c.skin;
    std::vector<float4> D, Dlo;
    if ((st = setup_grid(c, *box, D, Dlo)) != AP_OK) return fail(st);

    // region and indenter
    ap::DynDev& dy = c.dyn;
    std::memset(&dy, 0, sizeof(dy));
    c.region_kind = region ? region->kind : AP_REGION_NONE;
    dy.reg_kind = c.region_kind;
    if (region) {
        if (region->kind < 0 || region->kind > AP_REGION_CONST) { c.err = "bad region kind"; return fail(AP_ERR_ARG); }
        for (int k = 0; k < 3; ++k) dy.reg_c0[k] = region->center[k];
        dy.r_in = region->r_in;
        dy.r_sw = region->r_switch;
        dy.w_const = region->w_const;
        dy.follow = region->follow_indenter;
        if (region->kind == AP_REGION_SPHERE && !(region->r_switch > 0.0 && region->r_in >= 0.0)) { c.err = "sphere needs r_in >= 0, r_switch > 0"; return fail(AP_ERR_ARG); }
        if (region->kind == AP_REGION_CONST && !(region->w_const >= 0.0 && region->w_const <= 1.0)) { c.err = "w_const must lie in [0, 1]"; return fail(AP_ERR_ARG); }
        if (region->kind == AP_REGION_EXPLICIT && !region->w_explicit) { c.err = "explicit region needs w_explicit"; return fail(AP_ERR_ARG); }
    }
    if (ind && ind->enabled) {
        dy.ind_on = 1;
        for (int k = 0; k < 3; ++k) { dy.ind_c0[k] = ind->center0[k]; dy.ind_vel[k] = ind->vel[k]; dy.ind_dir[k] = ind->dir[k]; }
        dy.R = ind->R;
        dy.K = ind->K;
    }
    {
        const double ri = dy.r_in * (1.0 - 1e-5), ro = (dy.r_in + dy.r_sw) * (1.0 + 1e-5), rr = dy.R * (1.0 + 1e-5);
        dy.reg_in2_lo = (float)(ri * ri);
        dy.reg_out2_hi = (float)(ro * ro);
        dy.ind_R2_hi = (float)(rr * rr);
    }

    // device memory
    const size_t N = (size_t)n;
    c.nred = (n + ap::kRedBlock - 1) / ap::kRedBlock;
    {
        ArenaPlan plan;
        plan.add(&c.eam_d, 1); plan.add(&c.desc_d, 1); plan.add(&c.D, 125); plan.add(&c.Dlo, 125);
        plan.add(&c.pos_lo, N); plan.add(&c.x, 3 * N); plan.add(&c.v, 3 * N); plan.add(&c.xb, 3 * N);
        plan.add(&c.f, 3 * N); plan.add(&c.pos4, N); plan.add(&c.uxi, N); plan.add(&c.w, N);
        plan.add(&c.e_emb, N); plan.add(&c.e_eam, N); plan.add(&c.e_eam_acc, N); plan.add(&c.e_ace, N);
        plan.add(&c.ace_A, (size_t)ap::kNLM * ap::kNmax * N); plan.add(&c.ace_dA, (size_t)ap::kNLM * ap::kNmax * N);
        plan.add(&c.vir_eam, 6 * N); plan.add(&c.vir_ace, 6 * N); plan.add(&c.acc, 3 * N); plan.add(&c.fixed, N);
        plan.add(&c.w_fixed, N); plan.add(&c.cell, N); plan.add(&c.cell_atoms, N); plan.add(&c.nnbr, N);
        plan.add(&c.ace_list, N); plan.add(&c.flags, ap::kFlagCount); plan.add(&c.d_time, 1);
        plan.add(&c.partials, (size_t)c.nred * 10); plan.add(&c.totals, 16); plan.add(&c.e_atom, N);
        plan.add(&c.d_step, 1);
        // the cell arrays grow with the box (ap_set_box): allocated on their own
        if ((st = arena_commit(xc, plan)) || (st = dalloc(c, &c.cell_count, (size_t)c.grid.ncell)) ||
            (st = dalloc(c, &c.cell_start, (size_t)c.grid.ncell + 1)))
            return fail(st);
    }
    c.ncell_cap = c.grid.ncell;
    if (char* slot = pinned_take()) {
        c.h_totals = (double*)slot;
        c.h_flags = (int*)(slot + 16 * sizeof(double));
    } else {
        c.err = "pinned host allocation";
        return fail(AP_ERR_OOM);
    }
    // the host arrays go through a pinned staging block (pageable copies if none is had)
    const bool explicit_w = region && region->kind == AP_REGION_EXPLICIT;
    const size_t up_bytes = sizeof(ap::EamDev) + 2 * D.size() * sizeof(float4) + 2 * 3 * N * sizeof(double) +
                            (fixed ? N : 0) + (explicit_w ? N * sizeof(double) : 0) + 8 * 64;
    Staging stg;
    const bool staged = staging_take(up_bytes, c.dev, stg);
    struct StagingReturn {          // back to the pool on every path out of ap_init
        const Staging& b;
        cudaStream_t s;
        bool on;
        ~StagingReturn() { if (on) staging_give(b, s); }
    } stg_return{stg, c.stream, staged};
    size_t stg_used = 0;
    auto stage_copy = [&](const void* src, size_t bytes) -> const void* {
        if (!staged) return src;
        char* d = stg.p + stg_used;
        std::memcpy(d, src, bytes);
        stg_used += (bytes + 63) & ~(size_t)63;
        return d;
    };
    std::vector<double> soa;
    const double* pos_soa;
    const double* vel_soa = nullptr;
    if (staged) {
        double* d = (double*)(stg.p + stg_used);
        to_soa(pos, n, d);
        stg_used += (3 * N * sizeof(double) + 63) & ~(size_t)63;
        pos_soa = d;
        if (vel) {
            d = (double*)(stg.p + stg_used);
            to_soa(vel, n, d);
            stg_used += (3 * N * sizeof(double) + 63) & ~(size_t)63;
            vel_soa = d;
        }
    } else {
        to_soa(pos, n, soa);
        pos_soa = soa.data();
    }
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c.stream);
    };
    auto zero = [&](void* dst, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, bytes, c.stream);
    };
    cp(c.eam_d, stage_copy(&c.eam_h, sizeof(ap::EamDev)), sizeof(ap::EamDev));
    {
        std::unique_ptr<ap::AceTc> tc(new (std::nothrow) ap::AceTc());
        if (!tc) { c.err = "host allocation"; return fail(AP_ERR_OOM); }
        ap::build_ace_tc(*c.ace_h, *tc);
        c.ace_tc_d = ap::shared_ace_tables(*tc, c.dev, err);
        if (!c.ace_tc_d) { c.err = err; return fail(AP_ERR_OOM); }
    }
    cp(c.D, stage_copy(D.data(), D.size() * sizeof(float4)), D.size() * sizeof(float4));
    cp(c.Dlo, stage_copy(Dlo.data(), Dlo.size() * sizeof(float4)), Dlo.size() * sizeof(float4));
    cp(c.x, pos_soa, 3 * N * sizeof(double));
    cp(c.xb, pos_soa, 3 * N * sizeof(double));
    if (vel) {
        if (!staged) { to_soa(vel, n, soa); vel_soa = soa.data(); }
        cp(c.v, vel_soa, 3 * N * sizeof(double));
    } else {
        zero(c.v, 3 * N * sizeof(double));
    }
    if (fixed) cp(c.fixed, stage_copy(fixed, N), N);
    else zero(c.fixed, N);
    if (explicit_w) {
        for (int i = 0; i < n; ++i)
            if (!(region->w_explicit[i] >= 0.0 && region->w_explicit[i] <= 1.0)) { c.err = "explicit weights must lie in [0, 1]"; return fail(AP_ERR_ARG); }
        cp(c.w_fixed, stage_copy(region->w_explicit, N * sizeof(double)), N * sizeof(double));
    }
    zero(c.acc, 3 * N * sizeof(unsigned long long));
    zero(c.cell_count, (size_t)c.grid.ncell * sizeof(int));
    zero(c.flags, ap::kFlagCount * sizeof(int));
    zero(c.d_time, sizeof(double));
    zero(c.d_step, sizeof(long long));
    zero(c.vir_ace, 6 * N * sizeof(float));
    zero(c.e_ace, N * sizeof(float));
    zero(c.e_eam, N * sizeof(double));
    zero(c.e_eam_acc, N * sizeof(double));
    zero(c.e_emb, N * sizeof(double));
    zero(c.vir_eam, 6 * N * sizeof(float));
    int one = 1;
    cp(&c.flags[ap::kFlagRebuild], &one, sizeof(int));
    if (e != cudaSuccess) { cuda_check(c, e, "ap_init upload"); return fail(AP_ERR_CUDA); }

    cudaStream_t s = c.stream;
    if (pot->list_sizing == AP_LIST_BOUND) {
        // neighbour capacity from the density bound: nothing to wait for
        c.cap = list_capacity_bound(c.rc_list);
    } else {
        // size the neighbour capacity from a counting pass over the first binning
        c.launches += ap::launch_rebuild(c, s);
        c.launches += ap::launch_prepare(c, s);
        c.launches += ap::launch_build(c, s, 1);
        e = cudaMemcpyAsync(c.h_flags, c.flags, sizeof(int) * ap::kFlagCount, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) { cuda_check(c, e, "ap_init neighbour sizing"); return fail(AP_ERR_CUDA); }
        int need = c.h_flags[ap::kFlagMaxNbr];
        c.cap = std::max(8, ((int)(need * 1.25) + 8 + 3) & ~3);
    }
    if ((st = dalloc(c, &c.nbr, (size_t)c.cap * N)) || (st = dalloc(c, &c.nbr_tmp, (size_t)c.cap * N)) ||
        (st = dalloc(c, &c.nbr_row, (size_t)c.cap * N)))
        return fail(st);
    c.rebuilds = 0;
    *out = xc;
    return AP_OK;
}

ap_status ap_compute_forces(ap_ctx* xc, const double* d_pos, float* d_force, void* stream) {
    if (!xc) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    cudaStream_t s = pick(xc, stream);
    if (d_pos) c.launches += ap::launch_pos_in(c, s, d_pos);
    run_forces(xc, s, d_force);
    return cuda_check(c, cudaGetLastError(), "ap_compute_forces");
}

ap_status ap_compute_forces_host(ap_ctx* xc, const double* h_pos, float* h_force, double* h_energy, void* stream) {
    if (!xc) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    cudaStream_t s = pick(xc, stream);
    const size_t N = (size_t)c.n;
    ap_status st;
    if (!c.pos_stage && ((st = dalloc(c, &c.pos_stage, 3 * N)) || (st = dalloc(c, &c.f_stage, 3 * N)))) return st;
    cudaError_t e = cudaSuccess;
    if (capturable(s) && c.prof == 0) {
        // the kernels as one replayed graph
        const int mode = (h_pos ? 1 : 0) | (h_energy ? 2 : 0);
        if (xc->host_exec && (xc->host_stream != s || xc->host_gen != c.layout_gen || xc->host_mode != mode)) {
            cudaGraphExecDestroy(xc->host_exec);
            xc->host_exec = nullptr;
        }
        if (!xc->host_exec) {
            e = capture_graph(xc, s, &xc->host_exec, &xc->host_kernels, [&] {
                if (h_pos) c.launches += ap::launch_pos_in(c, s, c.pos_stage);
                run_forces(xc, s, c.f_stage, false, 0.0, h_energy != nullptr);   // with the energy blend
            });
            if (e != cudaSuccess) return graph_error(xc, e);
            xc->host_stream = s;
            xc->host_gen = c.layout_gen;
            xc->host_mode = mode;
        }
        if (h_pos) e = cudaMemcpyAsync(c.pos_stage, h_pos, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaGraphLaunch(xc->host_exec, s);
        if (e != cudaSuccess) return cuda_check(c, e, "ap_compute_forces_host");
        c.launches += xc->host_kernels;
        c.forces_valid = true;
        c.energy_fresh = h_energy != nullptr;
        if (h_energy) xc->energy_virial = false;
    } else {
        if (h_pos) {
            e = cudaMemcpyAsync(c.pos_stage, h_pos, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_check(c, e, "ap_compute_forces_host H2D");
            c.launches += ap::launch_pos_in(c, s, c.pos_stage);
        }
        // with every stage timed the EAM passes stay on s and the energy pass follows
        const bool branch_energy = h_energy && c.prof != 1;
        run_forces(xc, s, c.f_stage, false, 0.0, branch_energy);   // with the energy blend on the branch
        if (h_energy) {
            if (branch_energy) {                            // the total energy only
                c.energy_fresh = true;
                xc->energy_virial = false;
            } else {
                ensure_energy(xc, s, false);
                c.launches += ap::launch_reduce(c, s, 0);
            }
        }
    }
    if (h_force) e = cudaMemcpyAsync(h_force, c.f_stage, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_energy) e = cudaMemcpyAsync(c.h_totals, c.totals, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_compute_forces_host D2H");
    if ((st = read_flags(c, s))) return st;
    if (h_energy) *h_energy = c.h_totals[0] + c.h_totals[1];
    return AP_OK;
}

// the second half kick runs inside the force pass's blend kernel unless Langevin forces are
// added between them
static bool kick_in_blend(const ap::Ctx& c) { return c.thermo_kind != AP_THERMO_LANGEVIN; }

// the integration kernels around a force pass: part 0 before it (thermostat half step,
// kick-drift), part 1 after it (Langevin forces, kick, thermostat half step, momentum zeroing)
static int step_kernels(ap::Ctx& c, cudaStream_t s, double dt, int part) {
    int k = 0;
    if (part == 0) {
        if (c.thermo_kind == AP_THERMO_NOSE_HOOVER) k += ap::launch_nh_half(c, s, dt);
        k += ap::launch_kick_drift(c, s, dt, 1);
        return k;
    }
    if (c.thermo_kind == AP_THERMO_LANGEVIN) k += ap::launch_langevin(c, s, dt);
    if (!kick_in_blend(c)) k += ap::launch_kick(c, s, dt);
    if (c.thermo_kind == AP_THERMO_NOSE_HOOVER) k += ap::launch_nh_half(c, s, dt);
    if (c.thermo_kind == AP_THERMO_LANGEVIN && c.lv_zero_every > 0) k += ap::launch_zero_momentum(c, s);
    return k;
}


// The kernels of one captured MD step: kick-drift, the force pass, the kicks.  timed:
// event-record nodes of xc->ev_mark bracket the ACE contraction.
static void captured_step(ap_ctx* xc, cudaStream_t s, double dt, bool timed) {
    ap::Ctx& c = xc->c;
    const double kick = kick_in_blend(c) ? dt : 0.0;
    c.launches += step_kernels(c, s, dt, 0);
    if (!timed) {
        run_forces(xc, s, nullptr, true, kick);
    } else {
        run_forces_pre(xc, s, true);
        cudaError_t r = cudaEventRecordWithFlags(xc->ev_mark[0], s, cudaEventRecordExternal);
        c.launches += ap::launch_ace(c, s);
        if (r == cudaSuccess) r = cudaEventRecordWithFlags(xc->ev_mark[1], s, cudaEventRecordExternal);
        if (r != cudaSuccess && xc->cap_err == cudaSuccess) {
            xc->cap_err = r;
            xc->cap_where = "event record";
        }
        run_forces_post(xc, s, nullptr, kick, true);
    }
    c.launches += step_kernels(c, s, dt, 1);
}

// the timed step graph and the handles of its two event-record nodes
static cudaError_t capture_timed_step(ap_ctx* xc, cudaStream_t s, double dt) {
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 2 && e == cudaSuccess; ++q)
        if (!xc->ev_mark[q]) e = cudaEventCreate(&xc->ev_mark[q]);
    if (e == cudaSuccess)
        e = capture_graph(xc, s, &xc->timed_exec, &xc->timed_kernels, [&] { captured_step(xc, s, dt, true); },
                          &xc->timed_graph);
    if (e != cudaSuccess) return e;
    size_t nn = 0;
    e = cudaGraphGetNodes(xc->timed_graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(xc->timed_graph, nodes.data(), &nn);
    for (size_t k = 0; k < nn && e == cudaSuccess; ++k) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[k], &t);
        if (e != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        e = cudaGraphEventRecordNodeGetEvent(nodes[k], &ev);
        for (int q = 0; q < 2; ++q)
            if (ev == xc->ev_mark[q]) xc->ev_node[q] = nodes[k];
    }
    if (e == cudaSuccess && (!xc->ev_node[0] || !xc->ev_node[1])) {
        e = cudaErrorInvalidValue;
        xc->cap_where = "event nodes";
    }
    return e;
}

// one replay of the timed step graph with a fresh event pair on its event-record nodes
static cudaError_t replay_timed_step(ap_ctx* xc, cudaStream_t s) {
    if (xc->pending.size() >= 64) drain_ready(xc);
    cudaEvent_t a = get_event(xc), b = get_event(xc);
    cudaError_t e = cudaGraphExecEventRecordNodeSetEvent(xc->timed_exec, xc->ev_node[0], a);
    if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(xc->timed_exec, xc->ev_node[1], b);
    if (e == cudaSuccess) e = cudaGraphLaunch(xc->timed_exec, s);
    if (e == cudaSuccess) xc->pending.push_back({AP_STAGE_ACE, a, b});
    return e;
}

ap_status ap_step(ap_ctx* xc, int n_steps, double dt, void* stream) {
    if (!xc || n_steps < 0 || !(dt > 0.0)) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    cudaStream_t s = pick(xc, stream);
    if (!c.forces_valid) run_forces(xc, s, nullptr);
    if (c.prof == 1 || !capturable(s) || n_steps == 0) {
        const double kick = kick_in_blend(c) ? dt : 0.0;
        for (int k = 0; k < n_steps; ++k) {
            stage(xc, AP_STAGE_INTEGRATE, s, [&] { return step_kernels(c, s, dt, 0); });
            run_forces(xc, s, nullptr, true, kick);
            stage(xc, AP_STAGE_INTEGRATE, s, [&] { return step_kernels(c, s, dt, 1); });
            c.t += dt;
            c.step += 1;
        }
        return cuda_check(c, cudaGetLastError(), "ap_step");
    }
    if ((xc->step_exec || xc->block_exec || xc->timed_exec) &&
        (xc->step_stream != s || xc->step_dt != dt || xc->step_gen != c.layout_gen))
        drop_step_graph(xc);
    xc->step_stream = s;
    xc->step_dt = dt;
    xc->step_gen = c.layout_gen;
    // the graphs this call replays, captured on first need: the timed step (profiling modes
    // 2 and 3), the single step, the block of kStepBlock steps
    const bool timed = c.prof >= 2;
    const bool need_single = timed ? c.prof == 3 : n_steps % kStepBlock != 0;
    const bool need_block = !timed && n_steps >= kStepBlock;
    long long kernels = 0;
    cudaError_t e = cudaSuccess;
    if (timed && !xc->timed_exec) e = capture_timed_step(xc, s, dt);
    if (e == cudaSuccess && need_single && !xc->step_exec) {
        e = capture_graph(xc, s, &xc->step_exec, &kernels, [&] { captured_step(xc, s, dt, false); });
        if (e == cudaSuccess) xc->step_kernels = kernels;
    }
    if (e == cudaSuccess && need_block && !xc->block_exec) {
        e = capture_graph(xc, s, &xc->block_exec, &kernels, [&] {
            for (int q = 0; q < kStepBlock; ++q) captured_step(xc, s, dt, false);
        });
        if (e == cudaSuccess) xc->step_kernels = kernels / kStepBlock;
    }
    if (e != cudaSuccess) {
        drop_step_graph(xc);
        return graph_error(xc, e);
    }
    for (int left = n_steps; left > 0 && e == cudaSuccess;) {
        int k = 1;
        long long launched = xc->step_kernels;
        if (timed && (c.prof == 2 || (xc->timed_count++ & 7) == 0)) {
            // mode 3: one step in eight is timed, the others replay the untimed step graph
            e = replay_timed_step(xc, s);
            launched = xc->timed_kernels;
        } else if (!timed && left >= kStepBlock) {
            e = cudaGraphLaunch(xc->block_exec, s);
            k = kStepBlock;
        } else {
            e = cudaGraphLaunch(xc->step_exec, s);
        }
        c.launches += launched * k;
        c.t += dt * k;
        c.step += k;
        left -= k;
    }
    if (e != cudaSuccess) return cuda_check(c, e, "ap_step launch");
    c.forces_valid = true;
    c.energy_fresh = false;
    return AP_OK;
}

}  // extern "C"

namespace {

// the context's resident descriptor for batched launches, re-sent (on its own stream) when
// its contents changed: list capacity, box, load ring
void refresh_desc(ap_ctx* xc) {
    ap::Ctx& c = xc->c;
    ap::CtxDev d;
    ap::fill_ctx_dev(c, d);
    if (c.desc_valid && std::memcmp(c.desc_h, &d, sizeof(d)) == 0) return;
    std::memcpy(c.desc_h, &d, sizeof(d));
    cudaMemcpyAsync(c.desc_d, c.desc_h, sizeof(d), cudaMemcpyHostToDevice, c.stream);
    c.desc_valid = true;
}

// the batch table of a set of contexts: their descriptors and block prefixes
void batch_table(const std::vector<ap_ctx*>& cs, ap::BatchTable& t) {
    t.nctx = (int)cs.size();
    t.atoms = 0;
    t.b256[0] = t.b128[0] = t.bcell[0] = 0;
    for (int k = 0; k < t.nctx; ++k) {
        const ap::Ctx& c = cs[k]->c;
        t.d[k] = c.desc_d;
        t.b256[k + 1] = t.b256[k] + (c.n + 255) / 256;
        t.b128[k + 1] = t.b128[k] + (c.n + 127) / 128;
        t.bcell[k + 1] = t.bcell[k] + (c.grid.ncell + 7) / 8;          // a warp per cell, 8 per block
        t.atoms += c.n;
    }
}

// one AP force evaluation of every context of t, one launch per stage; kick_dt > 0: the
// blend applies the second half kick of a step (whose kick-drift ran the displacement test)
int batch_forces(const ap::BatchTable& t, int dev, cudaStream_t s, bool after_drift, double kick_dt) {
    int k = 0;
    if (!after_drift) k += ap::launch_batch_check(t, s);
    k += ap::launch_batch_rebuild(t, s);
    k += ap::launch_batch_prepare(t, s);
    k += ap::launch_batch_eam(t, s);
    k += ap::launch_batch_ace(t, dev, s);
    k += ap::launch_batch_blend(t, kick_dt, kick_dt > 0.0 ? 1 : 0, s);
    return k;
}

// contexts a batched launch can take: the plain step (no thermostat, no stage timing), the
// FP32 atomic base, the current device
bool batchable(const ap::Ctx& c, int dev) {
    return c.prof == 0 && c.thermo_kind == AP_THERMO_NONE && c.ace_prec == AP_ACE_FP32 && c.dev == dev;
}

// the batch stream waits for the contexts' earlier work
void batch_join_in(const std::vector<ap_ctx*>& cs, cudaStream_t bs) {
    for (ap_ctx* xc : cs) {
        refresh_desc(xc);
        cudaEvent_t e = get_event(xc);
        cudaEventRecord(e, xc->c.stream);
        cudaStreamWaitEvent(bs, e, 0);
        xc->free_ev.push_back(e);
    }
}

// the contexts' later work waits for the batch
void batch_join_out(const std::vector<ap_ctx*>& cs, cudaStream_t bs) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return;
    cudaEventRecord(e, bs);
    for (ap_ctx* xc : cs) cudaStreamWaitEvent(xc->c.stream, e, 0);
    cudaEventDestroy(e);
}

ap_status batch_status(const std::vector<ap_ctx*>& cs, cudaError_t e, const char* what) {
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) return AP_OK;
    ap_status st = AP_OK;
    for (ap_ctx* xc : cs) st = cuda_check(xc->c, e, what);
    return st;
}

// the batched form of ap_step for the contexts in cs (all batchable), with their step counts
ap_status batch_steps(std::vector<ap_ctx*> cs, std::vector<int> ns, double dt, cudaStream_t bs) {
    int dev = 0;
    cudaGetDevice(&dev);
    // contexts sharing a potential side by side: a block of the batched contraction then
    // stages coefficient tables only where the potential changes
    std::vector<int> order(cs.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return cs[a]->c.ace_tc_d < cs[b]->c.ace_tc_d; });
    std::vector<ap_ctx*> sc;
    std::vector<int> sn;
    for (int k : order) { sc.push_back(cs[k]); sn.push_back(ns[k]); }
    batch_join_in(sc, bs);
    std::unique_ptr<ap::BatchTable> t(new ap::BatchTable());
    std::vector<ap_ctx*> init;
    for (ap_ctx* xc : sc)
        if (!xc->c.forces_valid) init.push_back(xc);
    if (!init.empty()) {
        batch_table(init, *t);
        const int k = batch_forces(*t, dev, bs, false, 0.0);
        for (ap_ctx* xc : init) { xc->c.launches += k; xc->c.forces_valid = true; }
    }
    int maxs = 0;
    for (int v : sn) maxs = std::max(maxs, v);
    std::vector<ap_ctx*> active = sc;
    std::vector<int> left = sn;
    bool table = false;
    for (int st = 0; st < maxs; ++st) {
        // contexts whose steps are done leave the batch and are released to their own streams
        std::vector<ap_ctx*> now, done;
        std::vector<int> nl;
        for (size_t k = 0; k < active.size(); ++k) {
            if (left[k] > 0) { now.push_back(active[k]); nl.push_back(left[k]); }
            else done.push_back(active[k]);
        }
        if (!done.empty()) batch_join_out(done, bs);
        if (now.size() != active.size() || !table) {
            active = now;
            left = nl;
            batch_table(active, *t);
            table = true;
        }
        int k = ap::launch_batch_step_pre(*t, dt, bs);
        k += batch_forces(*t, dev, bs, true, dt);
        for (size_t q = 0; q < active.size(); ++q) {
            ap::Ctx& c = active[q]->c;
            c.launches += k;
            c.t += dt;
            c.step += 1;
            left[q] -= 1;
        }
    }
    for (ap_ctx* xc : sc) {
        xc->c.forces_valid = true;
        xc->c.energy_fresh = false;
    }
    batch_join_out(active, bs);
    return batch_status(sc, cudaSuccess, "batched step");
}

}  // namespace

extern "C" {

ap_status ap_step_batch(ap_ctx* const* ctxs, const int* n_steps, int n_ctx, double dt, void* stream) {
    if (!ctxs || !n_steps || n_ctx < 0 || !(dt > 0.0)) return AP_ERR_ARG;
    for (int k = 0; k < n_ctx; ++k)
        if (!ctxs[k] || n_steps[k] < 0) return AP_ERR_ARG;
    int dev = 0;
    cudaGetDevice(&dev);
    ap_status first = AP_OK;
    std::vector<ap_ctx*> bc;
    std::vector<int> bn;
    for (int k = 0; k < n_ctx; ++k) {
        if (n_steps[k] == 0) continue;
        if (batchable(ctxs[k]->c, dev) && (int)bc.size() < ap::kMaxBatchCtx) {
            bc.push_back(ctxs[k]);
            bn.push_back(n_steps[k]);
        } else {
            ap_status st = ap_step(ctxs[k], n_steps[k], dt, nullptr);
            if (st != AP_OK && first == AP_OK) first = st;
        }
    }
    if (!bc.empty()) {
        ap_status st = batch_steps(bc, bn, dt, (cudaStream_t)stream);
        if (st != AP_OK && first == AP_OK) first = st;
    }
    return first;
}

ap_status ap_compute_forces_batch(ap_ctx* const* ctxs, int n_ctx, void* stream) {
    if (!ctxs || n_ctx < 0) return AP_ERR_ARG;
    for (int k = 0; k < n_ctx; ++k)
        if (!ctxs[k]) return AP_ERR_ARG;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStream_t bs = (cudaStream_t)stream;
    ap_status first = AP_OK;
    std::vector<ap_ctx*> bc;
    for (int k = 0; k < n_ctx; ++k) {
        if (batchable(ctxs[k]->c, dev) && (int)bc.size() < ap::kMaxBatchCtx) {
            bc.push_back(ctxs[k]);
        } else {
            ap_status st = ap_compute_forces(ctxs[k], nullptr, nullptr, nullptr);
            if (st != AP_OK && first == AP_OK) first = st;
        }
    }
    if (!bc.empty()) {
        std::stable_sort(bc.begin(), bc.end(), [](ap_ctx* a, ap_ctx* b) { return a->c.ace_tc_d < b->c.ace_tc_d; });
        batch_join_in(bc, bs);
        std::unique_ptr<ap::BatchTable> t(new ap::BatchTable());
        batch_table(bc, *t);
        const int k = batch_forces(*t, dev, bs, false, 0.0);
        for (ap_ctx* xc : bc) {
            xc->c.launches += k;
            xc->c.forces_valid = true;
            xc->c.energy_fresh = false;
        }
        batch_join_out(bc, bs);
        ap_status st = batch_status(bc, cudaSuccess, "batched force evaluation");
        if (st != AP_OK && first == AP_OK) first = st;
    }
    return first;
}

ap_status ap_set_thermostat(ap_ctx* xc, const ap_thermostat* t, const unsigned char* group) {
    if (!xc || !t) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    if (t->kind != AP_THERMO_NONE && t->kind != AP_THERMO_NOSE_HOOVER && t->kind != AP_THERMO_LANGEVIN)
        return set_err(c, AP_ERR_ARG, "unknown thermostat kind");
    if (t->kind == AP_THERMO_LANGEVIN && t->zero_every < 0) return set_err(c, AP_ERR_ARG, "zero_every must be >= 0");
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_set_thermostat");
    drop_step_graph(xc);
    c.layout_gen += 1;                                   // the step graph changes shape
    if (t->kind == AP_THERMO_NONE) { c.thermo_kind = 0; return AP_OK; }
    if (!(t->t_target > 0.0) || !(t->tau_fs > 0.0)) return set_err(c, AP_ERR_ARG, "thermostat needs t_target > 0 and tau_fs > 0");
    const size_t N = (size_t)c.n;
    ap_status st;
    if (!c.thermo_group &&
        ((st = dalloc(c, &c.thermo_group, N)) || (st = dalloc(c, &c.nh_state, 4)) || (st = dalloc(c, &c.nh_partials, (size_t)c.nred)) ||
         (st = dalloc(c, &c.com, 4 * (size_t)c.nred + 4))))
        return st;
    std::vector<unsigned char> fx(N), g(N);
    e = cudaMemcpyAsync(fx.data(), c.fixed, N, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_set_thermostat");
    long long ng = 0;
    for (size_t i = 0; i < N; ++i) {
        g[i] = (group ? group[i] != 0 : true) && !fx[i];
        ng += g[i];
    }
    const double kB = 8.617333262e-5;
    c.nh_nfkt = 3.0 * (double)ng * kB * t->t_target;
    c.nh_Q = c.nh_nfkt * t->tau_fs * t->tau_fs;
    // Langevin: drag m/tau and noise sqrt(2 m k_B T / (tau dt)) in eV/A (dt enters at the step)
    c.lv_drag = c.mass / (t->tau_fs * ap::kFtm);
    c.lv_sig = 2.0 * c.mass * kB * t->t_target / (t->tau_fs * ap::kFtm);   // / dt, sqrt at the step
    c.lv_seed = t->seed;
    c.lv_zero_every = t->zero_every;
    c.lv_base = c.step;
    const double zero[4] = {0.0, 0.0, 1.0, 0.0};
    e = cudaMemcpyAsync(c.thermo_group, g.data(), N, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.nh_state, zero, sizeof(zero), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_set_thermostat");
    c.thermo_kind = ng > 0 ? t->kind : 0;
    return AP_OK;
}

static ap_status check_csp(ap::Ctx& c, const ap_csp_params* p) {
    if (!p || (p->n_nb != 12 && p->n_nb != 14)) return set_err(c, AP_ERR_ARG, "CSP: n_nb must be 12 or 14");
    if (!(p->rc > 0.0 && p->rc <= c.rc_list)) return set_err(c, AP_ERR_ARG, "CSP: rc must lie in (0, neighbour-list cutoff]");
    if (!(p->csp_hi > p->csp_lo) || !(p->r_hi > p->r_lo && p->r_lo >= 0.0) || !(p->dlam_min >= 0.0) || !(p->zone_r >= 0.0))
        return set_err(c, AP_ERR_ARG, "CSP: need csp_hi > csp_lo, r_hi > r_lo >= 0, dlam_min >= 0, zone_r >= 0");
    return AP_OK;
}

ap_status ap_csp_accumulate(ap_ctx* xc, const ap_csp_params* p, float* d_csp) {
    if (!xc) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    ap_status st;
    if ((st = check_csp(c, p))) return st;
    const size_t N = (size_t)c.n;
    if (!c.csp_sum) {
        if ((st = dalloc(c, &c.csp_sum, N)) || (st = dalloc(c, &c.csp_under, N)) || (st = dalloc(c, &c.csp_w0, N)) ||
            (st = dalloc(c, &c.csp_wnew, N)) || (st = dalloc(c, &c.csp_seeds, N)) || (st = dalloc(c, &c.csp_nseed, 1)))
            return st;
        cudaMemsetAsync(c.csp_sum, 0, N * sizeof(double), c.stream);
        cudaMemsetAsync(c.csp_under, 0, N * sizeof(int), c.stream);
        c.csp_nacc = 0;
    }
    if (!c.forces_valid) run_forces(xc, c.stream, nullptr);   // positions and list of the current state
    c.launches += ap::launch_csp(c, c.stream, *p, d_csp);
    c.csp_nacc += 1;
    return cuda_check(c, cudaGetLastError(), "ap_csp_accumulate");
}

ap_status ap_csp_update_weights(ap_ctx* xc, const ap_csp_params* p, int* n_seeds) {
    if (!xc) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    ap_status st;
    if ((st = check_csp(c, p))) return st;
    if (c.region_kind != AP_REGION_EXPLICIT) return set_err(c, AP_ERR_STATE, "CSP weights need an AP_REGION_EXPLICIT context");
    if (!c.csp_sum || c.csp_nacc == 0) return set_err(c, AP_ERR_STATE, "CSP: no evaluation in the current block");
    int S[3];
    for (int k = 0; k < 3; ++k) S[k] = std::max(1, (int)std::ceil(p->r_hi / c.grid.cw[k] - 1e-12));
    c.launches += ap::launch_csp_weights(c, c.stream, *p, c.csp_nacc, S);
    c.csp_nacc = 0;
    int ns = 0;
    cudaError_t e = cudaMemcpyAsync(&c.h_flags[ap::kFlagCount - 1], c.csp_nseed, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_csp_update_weights");
    ns = c.h_flags[ap::kFlagCount - 1];
    if (n_seeds) *n_seeds = ns;
    c.forces_valid = false;
    return AP_OK;
}

ap_status ap_energy(ap_ctx* xc, ap_report* out, double* d_e_atom) {
    if (!xc || !out) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    cudaStream_t s = c.stream;
    if (!c.forces_valid) run_forces(xc, s, nullptr);
    ensure_energy(xc, s);
    c.launches += ap::launch_reduce(c, s, 1);
    cudaError_t e = cudaMemcpyAsync(c.h_totals, c.totals, 10 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && c.thermo_kind)
        e = cudaMemcpyAsync(c.h_totals + 12, c.nh_state, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && d_e_atom)
        e = cudaMemcpyAsync(d_e_atom, c.e_atom, (size_t)c.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_energy");
    ap_status st = read_flags(c, s);
    std::memset(out, 0, sizeof(*out));
    const double* T = c.h_totals;
    out->e_pot = T[0];
    out->e_ind = T[1];
    out->e_total = T[0] + T[1];
    for (int k = 0; k < 6; ++k) out->virial[k] = T[2 + k];
    out->load = T[8];
    out->e_thermostat = c.thermo_kind ? 0.5 * c.nh_Q * T[12] * T[12] + c.nh_nfkt * T[13] : 0.0;
    out->e_kin = T[9];
    out->time_fs = c.t;
    out->step = c.step;
    out->n_ace = c.h_flags[ap::kFlagNAce];
    out->n_atoms = c.n;
    return st;
}

ap_status ap_check(ap_ctx* xc) {
    if (!xc) return AP_ERR_ARG;
    return read_flags(xc->c, xc->c.stream);
}

ap_status ap_get_state(ap_ctx* xc, double* x, double* v, double* t) {
    if (!xc) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    const size_t N = (size_t)c.n;
    std::vector<double> tmp(3 * N);
    for (int which = 0; which < 2; ++which) {
        double* dst = which == 0 ? x : v;
        if (!dst) continue;
        cudaError_t e = cudaMemcpyAsync(tmp.data(), which == 0 ? c.x : c.v, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) return cuda_check(c, e, "ap_get_state");
        for (size_t i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) dst[3 * i + k] = tmp[(size_t)k * N + i];
    }
    if (t) *t = c.t;
    return AP_OK;
}

ap_status ap_set_state(ap_ctx* xc, const double* x, const double* v, double t) {
    if (!xc) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    const size_t N = (size_t)c.n;
    std::vector<double> soa;
    cudaError_t e = cudaStreamSynchronize(c.stream);
    std::vector<double> soa_v;
    if (x && e == cudaSuccess) { to_soa(x, c.n, soa); e = cudaMemcpyAsync(c.x, soa.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice, c.stream); }
    if (v && e == cudaSuccess) { to_soa(v, c.n, soa_v); e = cudaMemcpyAsync(c.v, soa_v.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice, c.stream); }
    int one = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c.flags[ap::kFlagRebuild], &one, sizeof(int), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_time, &t, sizeof(double), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_set_state");
    c.t = t;
    c.forces_valid = false;
    return AP_OK;
}

ap_status ap_set_box(ap_ctx* xc, const ap_box* box) {
    if (!xc || !box) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_set_box");
    const ap::GridDev old = c.grid;
    std::vector<float4> D, Dlo;
    ap_status st = setup_grid(c, *box, D, Dlo);
    if (st != AP_OK) { c.grid = old; return st; }
    if (c.grid.ncell > c.ncell_cap) {
        int *cc = nullptr, *cs = nullptr;
        if (cudaMallocAsync((void**)&cc, (size_t)c.grid.ncell * sizeof(int), c.stream) != cudaSuccess ||
            cudaMallocAsync((void**)&cs, ((size_t)c.grid.ncell + 1) * sizeof(int), c.stream) != cudaSuccess) {
            if (cc) cudaFreeAsync(cc, c.stream);
            c.grid = old;
            return set_err(c, AP_ERR_OOM, "ap_set_box: cell arrays");
        }
        cudaFreeAsync(c.cell_count, c.stream);
        cudaFreeAsync(c.cell_start, c.stream);
        c.dev_bytes += 2 * ((size_t)c.grid.ncell - (size_t)c.ncell_cap) * sizeof(int);
        c.cell_count = cc;
        c.cell_start = cs;
        c.ncell_cap = c.grid.ncell;
    }
    e = cudaMemsetAsync(c.cell_count, 0, (size_t)c.grid.ncell * sizeof(int), c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.D, D.data(), D.size() * sizeof(float4), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.Dlo, Dlo.data(), Dlo.size() * sizeof(float4), cudaMemcpyHostToDevice, c.stream);
    int one = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c.flags[ap::kFlagRebuild], &one, sizeof(int), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_set_box");
    c.forces_valid = false;
    c.layout_gen += 1;
    return AP_OK;
}

ap_status ap_get_forces(ap_ctx* xc, float* f) {
    if (!xc || !f) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    const size_t N = (size_t)c.n;
    std::vector<float> tmp(3 * N);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), c.f, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_get_forces");
    for (size_t i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) f[3 * i + k] = tmp[(size_t)k * N + i];
    return AP_OK;
}

ap_status ap_get_weights(ap_ctx* xc, double* w) {
    if (!xc || !w) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    std::vector<float> tmp((size_t)c.n);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), c.w, (size_t)c.n * sizeof(float), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_get_weights");
    for (int i = 0; i < c.n; ++i) w[i] = tmp[i];
    return AP_OK;
}

ap_status ap_set_weights(ap_ctx* xc, const double* w) {
    if (!xc || !w) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    if (c.region_kind != AP_REGION_EXPLICIT) return set_err(c, AP_ERR_STATE, "weights are explicit only for AP_REGION_EXPLICIT");
    for (int i = 0; i < c.n; ++i)
        if (!(w[i] >= 0.0 && w[i] <= 1.0)) return set_err(c, AP_ERR_ARG, "weights must lie in [0, 1]");
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.w_fixed, w, (size_t)c.n * sizeof(double), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    c.forces_valid = false;
    return cuda_check(c, e, "ap_set_weights");
}

ap_status ap_profile(ap_ctx* xc, int enable) {
    if (!xc) return AP_ERR_ARG;
    if (enable < 0 || enable > 3) return AP_ERR_ARG;
    xc->c.prof = enable;
    xc->timed_count = 0;
    return AP_OK;
}

ap_status ap_profile_read(ap_ctx* xc, double* ms, long long* launches) {
    if (!xc) return AP_ERR_ARG;
    drain_events(xc);
    for (int k = 0; k < AP_NSTAGE; ++k) {
        if (ms) ms[k] = xc->c.stage_ms[k];
        if (launches) launches[k] = xc->c.stage_n[k];
        xc->c.stage_ms[k] = 0.0;
        xc->c.stage_n[k] = 0;
    }
    return AP_OK;
}

long long ap_launch_count(const ap_ctx* xc) { return xc ? xc->c.launches : 0; }

ap_status ap_neighbor_info(ap_ctx* xc, int* capacity, long long* rebuilds) {
    if (!xc) return AP_ERR_ARG;
    ap_status st = read_flags(xc->c, xc->c.stream);
    if (capacity) *capacity = xc->c.cap;
    if (rebuilds) *rebuilds = xc->c.h_flags[ap::kFlagRebuilds] - 1;   // the sizing pass at ap_init is not counted
    return st;
}

void ap_inject_alloc_failures(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

ap_status ap_record_load(ap_ctx* xc, int capacity) {
    if (!xc || capacity < 0) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    if (capacity > 0 && !c.dyn.ind_on) return set_err(c, AP_ERR_STATE, "ap_record_load: the context has no indenter");
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_record_load");
    drop_step_graph(xc);
    c.layout_gen += 1;                                   // the step kernels' arguments change
    if (c.load_ring) {
        cudaFreeAsync(c.load_ring, c.stream);
        cudaFreeAsync(c.load_ring_t, c.stream);
        c.dev_bytes -= (size_t)c.load_cap * (sizeof(long long) + sizeof(double));
        c.load_ring = nullptr;
        c.load_ring_t = nullptr;
        c.load_cap = 0;
    }
    if (capacity == 0) return AP_OK;
    ap_status st;
    if ((st = dalloc(c, &c.load_ring, (size_t)capacity)) || (st = dalloc(c, &c.load_ring_t, (size_t)capacity))) {
        if (c.load_ring) { cudaFreeAsync(c.load_ring, c.stream); c.dev_bytes -= (size_t)capacity * sizeof(long long); }
        c.load_ring = nullptr;
        return st;
    }
    c.load_cap = capacity;
    c.load_step0 = c.step;
    return AP_OK;
}

ap_status ap_load_history(ap_ctx* xc, double* t_fs, double* load, int max, int* count) {
    if (!xc || max < 0 || (max > 0 && (!t_fs || !load)) || !count) return AP_ERR_ARG;
    ap::Ctx& c = xc->c;
    *count = 0;
    if (!c.load_ring) return set_err(c, AP_ERR_STATE, "ap_load_history: no load history is recorded");
    const long long have = std::min<long long>(c.step - c.load_step0, c.load_cap);
    const int m = (int)std::min<long long>(have, max);
    std::vector<long long> ring((size_t)c.load_cap);
    std::vector<double> tt((size_t)c.load_cap);
    cudaError_t e = cudaMemcpyAsync(ring.data(), c.load_ring, ring.size() * sizeof(long long), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tt.data(), c.load_ring_t, tt.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_check(c, e, "ap_load_history");
    for (int k = 0; k < m; ++k) {
        const long long step = c.step - m + 1 + k;
        const size_t slot = (size_t)(step % c.load_cap);
        t_fs[k] = tt[slot];
        load[k] = (double)ring[slot] / ap::kLoadScale;
    }
    *count = m;
    return AP_OK;
}

const char* ap_last_error(const ap_ctx* xc) { return xc ? xc->c.err.c_str() : g_init_err.c_str(); }

void ap_destroy(ap_ctx* xc) {
    if (!xc) return;
    cudaStreamSynchronize(xc->c.stream);
    drop_step_graph(xc);
    for (cudaEvent_t e : xc->ev_mark)
        if (e) cudaEventDestroy(e);
    drain_events(xc);
    for (cudaEvent_t e : xc->free_ev) cudaEventDestroy(e);
    free_all(xc);
    delete xc;
}

ap_status ap_gaunt_real(int l1, int m1, int l2, int m2, int l3, int m3, double* out) {
    if (!out || l1 < 0 || l2 < 0 || l3 < 0 || l1 > 4 || l2 > 4 || l3 > 4) return AP_ERR_ARG;
    if (std::abs(m1) > l1 || std::abs(m2) > l2 || std::abs(m3) > l3) return AP_ERR_ARG;
    *out = ap::gaunt_real_racah(l1, m1, l2, m2, l3, m3);
    return AP_OK;
}

ap_status ap_eam_table_eval(const ap_potential* pot, int which, double r, double* f, double* df) {
    if (!pot || !f || !df || which < 0 || which > 3) return AP_ERR_ARG;
    return (ap_status)ap::eam_table_eval(*pot, which, r, f, df);
}

}  // extern "C"
