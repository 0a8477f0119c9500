// C ABI of the library and the host side of the Levenberg-Marquardt loop
// (Sec. 6.1): lambda0, the iteration limit, the relative function tolerance
// and the accept/reject rule with Nielsen's damping update.  The host only
// reads back a few scalars per LM iteration (the PCG scalars, the FP64 model
// cost and the FP64 candidate cost); everything else stays on the device.
#include <algorithm>
#include <map>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <memory>
#include <vector>

#include "camera.cuh"
#include "learned.cuh"
#include "problem.cuh"

namespace sqrtba {
int linearize_k_limit();

cudaMemPool_t device_pool() {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    BA_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    cudaMemPool_t& pool = pools[dev];
    if (!pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        BA_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = UINT64_MAX;  // never return freed memory to the system on synchronisation
        BA_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    return pool;
}

static std::mutex pinned_mu;
static std::multimap<size_t, void*> pinned_free;

void* pinned_get(size_t bytes) {
    {
        std::lock_guard<std::mutex> lock(pinned_mu);
        auto it = pinned_free.find(bytes);
        if (it != pinned_free.end()) {
            void* ptr = it->second;
            pinned_free.erase(it);
            return ptr;
        }
    }
    void* ptr = nullptr;
    BA_CUDA_TRY(cudaMallocHost(&ptr, bytes));
    return ptr;
}

void pinned_put(void* ptr, size_t bytes) {
    if (!ptr) return;
    std::lock_guard<std::mutex> lock(pinned_mu);
    pinned_free.emplace(bytes, ptr);
}

}  // namespace sqrtba

using namespace sqrtba;

struct ba_problem {
    Problem p;
};

struct ba_mlp {
    Mlp m;
};

struct ba_batch {
    Problem p;
    float* init_cams = nullptr;  // initial state (device), for ba_batch_restart
    float* init_pts = nullptr;
};

namespace {

thread_local std::string g_create_error;
constexpr int PCG_CHUNK = 8;

void set_error(ba_problem* h, const std::string& m) {
    if (h) h->p.last_error = m;
    else g_create_error = m;
}

#define API_TRY try {
#define API_CATCH(h)                                                      \
    }                                                                     \
    catch (const Error& e) {                                              \
        set_error(h, e.msg);                                              \
        return e.code;                                                    \
    }                                                                     \
    catch (const std::bad_alloc&) {                                       \
        set_error(h, "host allocation failed");                           \
        return BA_ERR_OOM;                                                \
    }                                                                     \
    catch (...) {                                                         \
        set_error(h, "unexpected exception");                             \
        return BA_ERR_CUDA;                                               \
    }

void require(bool cond, ba_status code, const char* msg) {
    if (!cond) throw Error{code, msg};
}

template <typename T>
void h2d(Problem& p, T* dst, const T* src, int64_t n) {
    BA_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, p.stream));
    p.h2d_bytes += (int64_t)sizeof(T) * n;
}
template <typename T>
void d2h(Problem& p, T* dst, const T* src, int64_t n) {
    BA_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyDeviceToHost, p.stream));
    p.d2h_bytes += (int64_t)sizeof(T) * n;
}
// device -> host copy that completes before returning (set-up only)
template <typename T>
void d2h_sync_copy(Problem& p, T* dst, const T* src, int64_t n) {
    BA_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyDeviceToHost, p.stream));
    BA_CUDA_TRY(cudaStreamSynchronize(p.stream));
}

// --- optional phase timing (CUDA events, resolved at synchronisation points) --
cudaEvent_t prof_event(Problem& p) {
    Profiler& f = p.prof;
    if (f.next == f.events.size()) {
        cudaEvent_t e;
        BA_CUDA_TRY(cudaEventCreate(&e));
        f.events.push_back(e);
    }
    return f.events[f.next++];
}

struct PhaseTimer {
    Problem& p;
    int slot;
    cudaEvent_t a = nullptr, b = nullptr;
    PhaseTimer(Problem& pp, int s) : p(pp), slot(s) {
        if (!p.prof.on) return;
        a = prof_event(p);
        b = prof_event(p);
        BA_CUDA_TRY(cudaEventRecord(a, p.stream));
    }
    void end() {
        if (!a) return;
        BA_CUDA_TRY(cudaEventRecord(b, p.stream));
        p.prof.pending.push_back({a, b, slot});
        a = nullptr;
    }
};

void prof_resolve(Problem& p) {
    Profiler& f = p.prof;
    for (auto& e : f.pending) {
        float ms = 0.f;
        BA_CUDA_TRY(cudaEventElapsedTime(&ms, e.a, e.b));
        f.ms[e.slot] += ms;
        f.count[e.slot] += 1;
    }
    f.pending.clear();
    f.next = 0;
}

void sync(Problem& p) {
    BA_CUDA_TRY(cudaStreamSynchronize(p.stream));
    if (p.prof.on) prof_resolve(p);
}

// The error words copied back with the last synchronisation (err_host): a
// bounded device wait that gave up (ERRBIT_TIMEOUT from the matvec / record
// pass, or from the attached model's tensor-core waits in err_host[3]) fails
// the call with BA_ERR_TIMEOUT; the counts of preconditioner blocks replaced
// by their diagonal and of cameras whose blocks were summed from the stored
// blocks are kept for the reports.  Words that were set are cleared on the
// device, in stream order, so that the handle stays usable.
void check_device_errors(Problem& p) {
    uint32_t* e = p.err_host;
    p.precond_fallbacks = (int32_t)e[1];
    p.precond_exact = (int32_t)e[2];
    const bool timeout = ((e[0] | e[3]) & ERRBIT_TIMEOUT) != 0;
    if (e[0] || e[1] || e[2]) BA_CUDA_TRY(cudaMemsetAsync(p.err, 0, 3 * sizeof(uint32_t), p.stream));
    if (e[3] && p.mlp) BA_CUDA_TRY(cudaMemsetAsync(p.mlp->err, 0, sizeof(uint32_t), p.stream));
    e[0] = e[1] = e[2] = e[3] = 0;
    if (timeout)
        throw Error{BA_ERR_TIMEOUT,
                    "a bounded device-side wait gave up; the kernel returned early and the results of this call "
                    "are invalid"};
}

// Synchronises with the error words copied back first, then checks them.
void sync_checked(Problem& p) {
    d2h(p, p.err_host, p.err, 3);
    if (p.mlp && p.learned_active) d2h(p, p.err_host + 3, p.mlp->err, 1);
    sync(p);
    check_device_errors(p);
}

void destroy_graph(Problem& p) {
    if (p.pcg_graph) cudaGraphExecDestroy(p.pcg_graph);
    p.pcg_graph = nullptr;
}

void free_all(Problem& p) {
    destroy_graph(p);
    for (cudaEvent_t e : p.batch.iter_events) cudaEventDestroy(e);
    p.batch.iter_events.clear();
    pinned_put(p.batch.n_active_host, sizeof(int32_t));
    p.batch.n_active_host = nullptr;
    for (cudaEvent_t e : p.prof.events) cudaEventDestroy(e);
    for (cudaEvent_t e : p.mv_events) cudaEventDestroy(e);
    p.prof.events.clear();
    p.mv_events.clear();
    for (void* a : p.allocations) cudaFreeAsync(a, p.stream);
    p.allocations.clear();
    pinned_put(p.pcg_host, sizeof(PcgScalars));
    pinned_put(p.dsum_host, 6 * sizeof(double));
    p.pcg_host = nullptr;
    p.dsum_host = nullptr;
    p.err_host = nullptr;
    if (p.side) cudaStreamDestroy(p.side);
    for (cudaEvent_t e : {p.ev_fork, p.ev_join})
        if (e) cudaEventDestroy(e);
    p.side = nullptr;
    p.ev_fork = p.ev_join = nullptr;
    if (p.own_stream && p.stream) cudaStreamDestroy(p.stream);
    p.stream = nullptr;
}

// --- the steps of the hot path ------------------------------------------------
// K1 (+ D_p^2).  The energy at the linearisation point is evaluated unless
// the host already knows it (the accepted candidate's cost).
// defer_cost: the energy is left in dsum[2] for the caller's next
// synchronisation (cost_pending) instead of being read back here.
void do_linearize(Problem& p, bool need_cost = true, double damp_lambda = 0.0, bool defer_cost = false) {
    const bool want_cost = need_cost || !p.cost_valid;
    PhaseTimer t(p, PROF_LINEARIZE);
    launch_frames(p);
    launch_linearize(p, want_cost ? (defer_cost ? 2 : 0) : -1);  // the energy beside K1
    t.end();
    if (damp_lambda > 0.0) {
        PhaseTimer td(p, PROF_DAMP);
        launch_damp(p, false, (float)damp_lambda);
        td.end();
    }
    if (want_cost) {
        if (defer_cost) {
            p.cost_pending = true;
            p.cost_valid = false;
        } else {
            d2h(p, p.dsum_host, p.dsum, 1);
            sync_checked(p);
            p.cost = p.dsum_host[0];
            p.cost_valid = true;
        }
    }
    p.linearized = true;
    p.damped = damp_lambda > 0.0;
    p.lambda_damped = damp_lambda;
    p.solved = false;
    p.backsubbed = false;
}

void do_marginalize(Problem& p, double lambda) {
    require(p.linearized, BA_ERR_STATE, "ba_marginalize_qr: problem is not linearised");
    require(std::isfinite(lambda) && lambda > 0.0, BA_ERR_INVALID_ARG, "lambda must be positive and finite");
    PhaseTimer t(p, PROF_DAMP);
    launch_damp(p, p.damped, (float)lambda);
    t.end();
    p.damped = true;
    p.lambda_damped = lambda;
    p.solved = false;
    p.backsubbed = false;
}

cudaEvent_t mv_event(Problem& p, int i) {
    return p.prof.on ? p.mv_events[i] : nullptr;
}

void capture_pcg_graph(Problem& p) {
    cudaGraph_t graph = nullptr;
    BA_CUDA_TRY(cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal));
    p.capturing = true;
    try {
        for (int i = 0; i < PCG_CHUNK; ++i) launch_pcg_iteration(p, mv_event(p, 2 * i), mv_event(p, 2 * i + 1));
    } catch (...) {
        p.capturing = false;
        cudaStreamEndCapture(p.stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    p.capturing = false;
    BA_CUDA_TRY(cudaStreamEndCapture(p.stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&p.pcg_graph, graph, 0);
    cudaGraphDestroy(graph);
    BA_CUDA_TRY(e);
    p.pcg_graph_iters = PCG_CHUNK;
}

// The whole CG as one graph launch: a conditional WHILE node whose body is
// one iteration (matvec + update); the update kernel clears the condition
// when a stop rule fires (the iteration limit bounds the loop).  Event
// record nodes are not allowed in conditional bodies, so profiling runs use
// the chunked graph above.
void capture_pcg_while_graph(Problem& p) {
    cudaGraph_t graph = nullptr;
    BA_CUDA_TRY(cudaGraphCreate(&graph, 0));
    try {
        cudaGraphConditionalHandle cond;
        BA_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams prm = {};
        prm.type = cudaGraphNodeTypeConditional;
        prm.conditional.handle = cond;
        prm.conditional.type = cudaGraphCondTypeWhile;
        prm.conditional.size = 1;
        cudaGraphNode_t node;
        BA_CUDA_TRY(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &prm));
        cudaGraph_t body = prm.conditional.phGraph_out[0];
        BA_CUDA_TRY(cudaStreamBeginCaptureToGraph(p.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        p.capturing = true;
        try {
            launch_pcg_iteration(p, nullptr, nullptr, true, cond);
        } catch (...) {
            p.capturing = false;
            cudaGraph_t g2 = nullptr;
            cudaStreamEndCapture(p.stream, &g2);
            throw;
        }
        p.capturing = false;
        cudaGraph_t g2 = nullptr;
        BA_CUDA_TRY(cudaStreamEndCapture(p.stream, &g2));
        BA_CUDA_TRY(cudaGraphInstantiate(&p.pcg_graph, graph, 0));
    } catch (...) {
        cudaGraphDestroy(graph);
        throw;
    }
    cudaGraphDestroy(graph);
    p.pcg_graph_iters = 0;  // the graph runs the CG to its end
}

// --- matvec autotuner ----------------------------------------------------------
struct EventSet {
    std::vector<cudaEvent_t> ev;
    explicit EventSet(int n) : ev(n, nullptr) {
        for (auto& e : ev) BA_CUDA_TRY(cudaEventCreate(&e));
    }
    ~EventSet() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
};

// median of five timed launches of the matvec (pc = false) or of the
// preconditioner record pass (pc = true) with the plan (ksmall, bytes) at
// pipeline depth ns (y in shared memory where y_smem and it fits)
double time_plan(Problem& p, bool pc, int ksmall, int bytes, int ns, int y_smem, EventSet& es, int big8 = -1) {
    Problem::TilePlan& plan = pc ? p.pc_plan : p.mv_plan;
    if (big8 >= 0) plan.big8_kmax = big8;
    if (plan.ksmall != ksmall || plan.small_bytes != bytes || plan.n == 0) {
        plan.ksmall = ksmall;
        plan.small_bytes = bytes;
        plan_tiles(p, pc);
    }
    plan.ns = ns;
    plan.y_smem = y_smem;
    count_launches(p, 6);
    auto run = [&] {
        if (pc) launch_precond_records(p);
        else launch_matvec_raw(p, p.p, p.q, nullptr);
    };
    run();
    for (int i = 0; i < 5; ++i) {
        BA_CUDA_TRY(cudaEventRecord(es.ev[2 * i], p.stream));
        run();
        BA_CUDA_TRY(cudaEventRecord(es.ev[2 * i + 1], p.stream));
    }
    BA_CUDA_TRY(cudaStreamSynchronize(p.stream));
    std::vector<float> t(5);
    for (int i = 0; i < 5; ++i) BA_CUDA_TRY(cudaEventElapsedTime(&t[i], es.ev[2 * i], es.ev[2 * i + 1]));
    std::sort(t.begin(), t.end());
    return t[2];
}

// Times every plan (ksmall in {8, 13, 21} x small_bytes in {8, 16, 32} KB)
// for the matvec and for the record pass at the default depth (6 stages, y
// in shared memory where it fits), keeps the fastest of each, then times that
// plan at depths 4, 5 and 6 (the matvec also with y in global memory) and
// keeps the fastest depth; last, for a matvec plan with row tiles, the
// largest k whose row tiles take eight rows a warp (0, 32, 40, 64, all).
void run_autotune(Problem& p, ba_tune_report* rep) {
    require(p.damped, BA_ERR_STATE, "ba_autotune: blocks are not marginalised (call ba_marginalize_qr)");
    require(!p.implicit, BA_ERR_INVALID_ARG, "ba_autotune: the tile plans apply to the stored blocks only");
    const auto t0 = std::chrono::steady_clock::now();
    EventSet es(10);
    // a non-zero input (D_p^2), so that the timed launches do the work of a
    // CG iteration (zero contributions skip the flush of y)
    BA_CUDA_TRY(cudaMemcpyAsync(p.p, p.dp2, sizeof(float) * 9 * p.n_cam, cudaMemcpyDeviceToDevice, p.stream));
    const int ks_opts[3] = {8, 13, 21};
    const int by_opts[3] = {8192, 16384, 32768};
    const Problem::TilePlan dflt{};
    p.mv_plan.big8_kmax = dflt.big8_kmax;
    double def = 0.0;
    if (rep) {  // the record pass's plan as it stands (replaced below when it is tuned)
        rep->pc_ksmall = p.pc_plan.ksmall;
        rep->pc_small_bytes = p.pc_plan.small_bytes;
        rep->pc_ns = p.opt.pipeline_stages ? p.opt.pipeline_stages : p.pc_plan.ns;
    }
    // the record pass runs only when the blocks are summed from A_j
    for (int pc = 0; pc < (p.opt.precond_from_blocks ? 2 : 1); ++pc) {
        double best = time_plan(p, pc, dflt.ksmall, dflt.small_bytes, dflt.ns, 1, es);
        if (!pc) def = best;
        int best_ks = dflt.ksmall, best_by = dflt.small_bytes;
        for (int ks : ks_opts)
            for (int by : by_opts) {
                if (ks == dflt.ksmall && by == dflt.small_bytes) continue;
                const double t = time_plan(p, pc, std::min(ks, matvec_ksmall_limit()), by, dflt.ns, 1, es);
                if (t < best) {
                    best = t;
                    best_ks = ks;
                    best_by = by;
                }
            }
        int best_ns = dflt.ns, best_y = 1;
        for (int ns = 4; ns <= 6 && p.opt.pipeline_stages == 0; ++ns)
            for (int y = pc ? 0 : 1; y >= 0; --y) {
                if (ns == dflt.ns && (y == 1 || pc)) continue;  // timed above
                const double t = time_plan(p, pc, best_ks, best_by, ns, y, es);
                if (t < best) {
                    best = t;
                    best_ns = ns;
                    best_y = y;
                }
            }
        // matvec row tiles: the largest k that takes eight rows a warp
        int best_b8 = dflt.big8_kmax;
        if (!pc && p.k_max > std::min(best_ks, matvec_ksmall_limit()))
            for (int b8 : {0, 32, 64, 1 << 20}) {
                const double t = time_plan(p, pc, best_ks, best_by, best_ns, best_y, es, b8);
                if (t < best) {
                    best = t;
                    best_b8 = b8;
                }
            }
        Problem::TilePlan& plan = pc ? p.pc_plan : p.mv_plan;
        plan.big8_kmax = best_b8;
        if (plan.ksmall != best_ks || plan.small_bytes != best_by) {
            plan.ksmall = best_ks;
            plan.small_bytes = best_by;
            plan_tiles(p, pc);
        }
        plan.ns = best_ns;
        plan.y_smem = best_y;
        if (rep && !pc) {
            rep->ksmall = best_ks;
            rep->small_bytes = best_by;
            rep->matvec_ms = best;
            rep->default_ms = def;
            rep->ns = p.opt.pipeline_stages ? p.opt.pipeline_stages : best_ns;
            rep->y_smem = matvec_y_in_smem(p) ? 1 : 0;
            rep->big8_kmax = best_b8;
        }
        if (rep && pc) {
            rep->pc_ksmall = best_ks;
            rep->pc_small_bytes = best_by;
            rep->pc_ns = p.opt.pipeline_stages ? p.opt.pipeline_stages : best_ns;
        }
    }
    destroy_graph(p);  // the captured launches hold the old plan
    p.tuned = true;
    const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) rep->tune_ms = wall;
}

// K8 before the CG: features of every camera, the MLP, the warm start x0
// (into x) and the corrected blocks B_i; q = (A^T A) x0 for the residual.
void start_learned(Problem& p) {
    if (!p.minv_l) {
        p.lfeat = dalloc<float>(p, (int64_t)ML_IN * p.n_cam);
        p.laux = dalloc<float>(p, (int64_t)ML_AUX * p.n_cam);
        p.minv_l = dalloc<float>(p, 81LL * p.n_cam);
    }
    learned_apply(p, *p.mlp);
    BA_CUDA_TRY(cudaMemsetAsync(p.q, 0, sizeof(float) * 9 * p.n_cam, p.stream));
    count_launches(p, 1);
    launch_matvec_raw(p, p.x, p.q, nullptr);
    launch_pcg_init_warm(p);
}

// K3 and the CG start (plain, or K8 with the learned warm start)
void pcg_start(Problem& p) {
    require(p.damped, BA_ERR_STATE, "ba_pcg_solve: blocks are not marginalised (call ba_marginalize_qr)");
    const bool learned = p.opt.use_learned != 0;
    require(!learned || p.mlp, BA_ERR_STATE, "use_learned is set but no model is attached (ba_set_learned)");
    require(!learned || p.batch.n_prob == 0, BA_ERR_INVALID_ARG, "the learned mode solves single problems");
    if (p.opt.autotune && !p.tuned) run_autotune(p, nullptr);
    PhaseTimer t(p, PROF_PRECOND);
    const bool fused = launch_precond_rhs(p, !learned);
    p.learned_active = learned;
    if (learned) start_learned(p);
    else if (!fused) launch_pcg_init(p);
    t.end();
}

// Runs the CG iterations.  The WHILE graph needs no host round trip: the
// scalars are copied back behind it and read at the next synchronisation
// (wait = true synchronises here).  The chunked forms (profiling, or no
// graphs) poll the done flag after every chunk of PCG_CHUNK iterations.
void pcg_iterate(Problem& p, bool wait) {
    const bool while_graph = p.opt.use_graph && !p.prof.on;
    const int kind = !p.opt.use_graph ? 0 : (while_graph ? 2 : 1);
    if (p.pcg_graph && (p.graph_learned != p.learned_active || p.graph_kind != kind)) destroy_graph(p);
    if (p.opt.use_graph && !p.pcg_graph) {
        if (while_graph) capture_pcg_while_graph(p);
        else capture_pcg_graph(p);
        p.graph_learned = p.learned_active;
        p.graph_kind = kind;
    }
    if (while_graph) {
        BA_CUDA_TRY(cudaGraphLaunch(p.pcg_graph, p.stream));
        count_launches(p, 2);  // per iteration; the rest is added when the count is known
        p.pending_iteration_launches = true;
        d2h(p, p.pcg_host, p.pcg, 1);
        if (wait) sync_checked(p);
        return;
    }
    int launched = 0, it_before = 0;
    for (;;) {
        if (p.opt.use_graph) {
            BA_CUDA_TRY(cudaGraphLaunch(p.pcg_graph, p.stream));
            count_launches(p, 2 * p.pcg_graph_iters);
        } else {
            for (int i = 0; i < PCG_CHUNK; ++i) launch_pcg_iteration(p, mv_event(p, 2 * i), mv_event(p, 2 * i + 1));
        }
        launched += PCG_CHUNK;
        d2h(p, p.pcg_host, p.pcg, 1);
        sync_checked(p);
        if (p.prof.on) {
            const int real = std::min(PCG_CHUNK, p.pcg_host->it - it_before);
            for (int i = 0; i < real; ++i) {
                float ms = 0.f;
                BA_CUDA_TRY(cudaEventElapsedTime(&ms, p.mv_events[2 * i], p.mv_events[2 * i + 1]));
                p.prof.ms[PROF_MATVEC] += ms;
                p.prof.count[PROF_MATVEC] += 1;
            }
        }
        it_before = p.pcg_host->it;
        if (p.pcg_host->done || launched >= p.opt.max_cg_iters + PCG_CHUNK) break;
    }
}

// After the CG's scalars are on the host: the learned solve is judged by the
// quadratic model of its iterate, Q(x) = -1/2 x^T (g + r) with r the
// recursion's residual; on a breakdown, or no decrease below Q(0) = 0, the
// plain block-Jacobi CG from zero is run instead.  Returns true if it re-ran.
bool pcg_judge(Problem& p) {
    if (p.pending_iteration_launches) {
        // the loop body ran max(it, 1) times (a batch: once more, to end the loop)
        count_launches(p, 2 * std::max(0, p.pcg_host->it - 1) + (p.batch.n_prob > 0 ? 2 : 0));
        p.pending_iteration_launches = false;
    }
    if (!(p.learned_active && (p.pcg_host->stop == 3 || !(p.pcg_host->q_prev < 0.f)))) return false;
    p.learned_active = false;
    p.learned_fallbacks += 1;
    launch_pcg_init(p);
    pcg_iterate(p, true);
    if (p.pending_iteration_launches) {
        count_launches(p, 2 * std::max(0, p.pcg_host->it - 1));
        p.pending_iteration_launches = false;
    }
    return true;
}

void fill_pcg_report(const Problem& p, ba_pcg_report* rep) {
    if (!rep) return;
    rep->iterations = p.pcg_host->it;
    rep->stop_reason = p.pcg_host->stop;
    rep->residual_norm = p.pcg_host->rnorm;
    rep->rhs_norm = p.pcg_host->gnorm;
    rep->learned = p.learned_active ? 1 : 0;
    rep->warm_start = p.learned_active ? p.pcg_host->warm : 0;
    rep->precond_fallbacks = p.precond_fallbacks;
    rep->precond_exact = p.precond_exact;
}

void do_pcg(Problem& p, ba_pcg_report* rep) {
    pcg_start(p);
    pcg_iterate(p, true);
    pcg_judge(p);
    p.solved = true;
    p.backsubbed = false;
    fill_pcg_report(p, rep);
}

double do_backsub(Problem& p) {
    require(p.solved, BA_ERR_STATE, "ba_backsubstitute: no PCG solution");
    PhaseTimer t(p, PROF_BACKSUB);
    launch_backsub(p);
    t.end();
    d2h(p, p.dsum_host + 1, p.dsum + 1, 1);
    sync_checked(p);
    p.backsubbed = true;
    return p.dsum_host[1];
}

double do_eval_cost(Problem& p, bool candidate) {
    if (candidate) {
        require(p.backsubbed, BA_ERR_STATE, "ba_eval_cost: no back-substituted step");
    }
    PhaseTimer t(p, PROF_COST);
    if (candidate) launch_candidate(p);
    launch_cost(p, candidate);
    t.end();
    d2h(p, p.dsum_host, p.dsum, 1);
    sync_checked(p);
    return p.dsum_host[0];
}

void do_lm_step(Problem& p, ba_lm_report* rep) {
    require(!p.stopped, BA_ERR_STATE, "ba_lm_step: the LM loop has stopped");
    ba_lm_report r{};
    r.iteration = p.iteration;
    const double lam = p.lambda;
    if (!p.linearized) {
        do_linearize(p, false, lam, true);  // an unknown energy is read back with the step's scalars
        r.relinearized = 1;
    }
    if (!p.damped || p.lambda_damped != lam) do_marginalize(p, lam);
    // K3-K7 enqueued back to back; one synchronisation for the scalars
    // (the learned mode synchronises once more to judge its CG)
    pcg_start(p);
    const bool learned = p.learned_active;
    pcg_iterate(p, learned);
    if (learned) pcg_judge(p);
    p.solved = true;
    {
        PhaseTimer tb(p, PROF_BACKSUB);
        launch_backsub_candidate_cost(p);
        tb.end();
    }
    // the scalars and, behind them in the same allocation, the error words
    d2h(p, p.dsum_host, p.dsum, 6);
    if (learned && p.mlp) d2h(p, p.err_host + 3, p.mlp->err, 1);
    sync(p);
    check_device_errors(p);
    if (p.cost_pending) {
        p.cost = p.dsum_host[2];
        p.cost_valid = true;
        p.cost_pending = false;
    }
    const double E = p.cost;
    if (!learned) pcg_judge(p);
    ba_pcg_report pr{};
    fill_pcg_report(p, &pr);
    p.backsubbed = true;
    const double L = p.dsum_host[1];
    const double En = p.dsum_host[0];
    // a step is accepted only if the model predicts a decrease (E - L > 0);
    // near convergence both differences sink below the FP32 evaluation noise
    // and their ratio alone would accept noise
    const double rho = (E - En) / (E - L);
    const bool acc = std::isfinite(En) && std::isfinite(rho) && (E - L) > 0.0 && rho > 1e-3;
    r.cost = E;
    r.new_cost = En;
    r.model_cost = L;
    r.lambda = lam;
    r.rho = rho;
    r.cg_iters = pr.iterations;
    r.pcg_stop_reason = pr.stop_reason;
    r.precond_fallbacks = pr.precond_fallbacks;
    r.precond_exact = pr.precond_exact;
    r.accepted = acc ? 1 : 0;
    if (acc) {
        std::swap(p.cams, p.cand_cams);
        std::swap(p.pts, p.cand_pts);
        std::swap(p.frames, p.cand_frames);
        p.cost = En;
        p.cost_valid = true;
        p.linearized = false;
        p.damped = false;
        p.solved = false;
        p.backsubbed = false;
        const double t = 2.0 * rho - 1.0;
        p.lambda *= std::max(1.0 / 3.0, 1.0 - t * t * t);
        p.lambda = std::max(p.lambda, 1e-16);
        p.nu = 2.0;
        if (std::fabs(E - En) / E < p.opt.func_tol) p.stopped = true;
        if (p.opt.target_cost > 0.0 && En <= p.opt.target_cost) p.stopped = true;
    } else {
        p.lambda *= p.nu;
        p.nu *= 2.0;
        if (p.lambda >= 1e32) {
            p.lambda = 1e32;
            p.stopped = true;
        }
    }
    p.iteration += 1;
    if (p.iteration >= p.opt.max_lm_iters) p.stopped = true;
    r.stop = p.stopped ? 1 : 0;
    if (rep) *rep = r;
}

// Allocates and fills a problem from host FP64 arrays: validation, grouping
// by landmark, storage and matvec plan, block pools.
void create_problem(Problem& p, const double* cams, int32_t n_cam, const double* pts, int32_t n_pt,
                    const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_xy, int64_t n_obs,
                    const ba_options* opt, void* cuda_stream) {
    require(cams && pts && obs_cam && obs_pt && obs_xy, BA_ERR_INVALID_ARG, "null input pointer");
    require(n_cam >= 1 && n_pt >= 1 && n_obs >= 2, BA_ERR_INVALID_ARG, "empty problem");
    require(n_obs < ((int64_t)1 << 31) - 1, BA_ERR_INVALID_ARG, "too many observations (limit 2^31 - 2)");
    ba_default_options(&p.opt);
    if (opt) p.opt = *opt;
    require(p.opt.lambda0 > 0 && p.opt.max_lm_iters >= 1 && p.opt.max_cg_iters >= 1 && p.opt.cg_eta > 0 &&
            (p.opt.pipeline_stages == 0 || (p.opt.pipeline_stages >= 4 && p.opt.pipeline_stages <= 6)) &&
            (p.opt.implicit_blocks == 0 || p.opt.implicit_blocks == 1) &&
            std::isfinite(p.opt.huber_delta) && p.opt.huber_delta >= 0.0 &&
            (p.opt.schur_explicit == 0 || (p.opt.schur_explicit == 1 && p.opt.implicit_blocks == 0)),
            BA_ERR_INVALID_ARG, "invalid options");
    p.implicit = p.opt.implicit_blocks != 0;
    p.schur = p.opt.schur_explicit != 0;
    p.n_cam = n_cam;
    p.n_pt = n_pt;
    p.n_obs = n_obs;
    p.lambda = p.opt.lambda0;
    p.nu = 2.0;
    if (cuda_stream) {
        p.stream = (cudaStream_t)cuda_stream;
    } else {
        BA_CUDA_TRY(cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking));
        p.own_stream = true;
    }
    BA_CUDA_TRY(cudaStreamCreateWithFlags(&p.side, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&p.ev_fork, &p.ev_join})
        BA_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    int dev = 0;
    BA_CUDA_TRY(cudaGetDevice(&dev));
    BA_CUDA_TRY(cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, dev));
    p.mv_grid = p.sm_count * matvec_ctas_per_sm();
    p.red_grid = p.sm_count * 4;

    p.cams = dalloc<float>(p, 9 * (int64_t)n_cam);
    p.cand_cams = dalloc<float>(p, 9 * (int64_t)n_cam);
    p.pts = dalloc<float>(p, 3 * (int64_t)n_pt);
    p.cand_pts = dalloc<float>(p, 3 * (int64_t)n_pt);
    p.frames = dalloc<float>(p, FRAME * (int64_t)n_cam);
    p.cand_frames = dalloc<float>(p, FRAME * (int64_t)n_cam);
    p.obs_cam_s = dalloc<int32_t>(p, n_obs);
    p.obs_pt_s = dalloc<int32_t>(p, n_obs);
    p.perm = dalloc<int32_t>(p, n_obs);
    p.obs_xy_s = dalloc<float2>(p, n_obs);
    p.pt_off = dalloc<int32_t>(p, n_pt + 1);
    p.cam_off = dalloc<int32_t>(p, n_cam + 1);
    p.cam_list = dalloc<int32_t>(p, n_obs);
    p.a_off = dalloc<int64_t>(p, n_pt + 1);
    p.lm_by_k = dalloc<int32_t>(p, n_pt);
    p.mv_cam = dalloc<int32_t>(p, n_obs + 8);
    p.c_off = dalloc<int32_t>(p, n_pt + 1);
    p.cam_list_st = dalloc<int32_t>(p, n_obs);
    // dsum [0..3] and the error words behind it: one copy brings back both
    p.dsum = dalloc<double>(p, 6);
    p.err = reinterpret_cast<uint32_t*>(p.dsum + 4);
    p.pcg = dalloc<PcgScalars>(p, 1);
    p.pcg_host = static_cast<PcgScalars*>(pinned_get(sizeof(PcgScalars)));
    p.dsum_host = static_cast<double*>(pinned_get(6 * sizeof(double)));
    p.err_host = reinterpret_cast<uint32_t*>(p.dsum_host + 4);
    std::memset(p.dsum_host, 0, 6 * sizeof(double));
    BA_CUDA_TRY(cudaMemsetAsync(p.dsum, 0, 6 * sizeof(double), p.stream));
    std::memset(p.pcg_host, 0, sizeof(PcgScalars));

    // stage the FP64 inputs on the device for validation and grouping
    double *d_cams = nullptr, *d_pts = nullptr, *d_xy = nullptr;
    int32_t *d_oc = nullptr, *d_op = nullptr;
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&d_cams, sizeof(double) * 9 * n_cam, device_pool(), p.stream));
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&d_pts, sizeof(double) * 3 * n_pt, device_pool(), p.stream));
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&d_xy, sizeof(double) * 2 * n_obs, device_pool(), p.stream));
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&d_oc, sizeof(int32_t) * n_obs, device_pool(), p.stream));
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&d_op, sizeof(int32_t) * n_obs, device_pool(), p.stream));
    struct StageGuard {
        Problem& p;
        void* b[5];
        ~StageGuard() {
            for (void* x : b)
                if (x) cudaFreeAsync(x, p.stream);
        }
    } sg{p, {d_cams, d_pts, d_xy, d_oc, d_op}};
    h2d(p, d_cams, cams, 9 * (int64_t)n_cam);
    h2d(p, d_pts, pts, 3 * (int64_t)n_pt);
    h2d(p, d_xy, obs_xy, 2 * n_obs);
    h2d(p, d_oc, obs_cam, n_obs);
    h2d(p, d_op, obs_pt, n_obs);
    build_index(p, d_oc, d_op, d_xy, d_cams, d_pts);
    require(p.k_max <= linearize_k_limit(), BA_ERR_INVALID_ARG,
            "a landmark has more observations than the supported maximum (900)");
    if (p.schur) {
        // the explicit Schur complement: its pattern from the sorted observations
        std::vector<int32_t> h_pt_off(n_pt + 1), h_cam(n_obs);
        d2h_sync_copy(p, h_pt_off.data(), p.pt_off, n_pt + 1);
        d2h_sync_copy(p, h_cam.data(), p.obs_cam_s, n_obs);
        plan_schur(p, h_pt_off, h_cam);
        p.tuned = true;
    } else if (!p.implicit) {  // the implicit storage keeps no top rows (landmark records instead)
        p.t_floats = 3 * (9 * n_obs + 4 * (int64_t)n_pt);
        p.tpool = dalloc<float>(p, p.t_floats);
    }
    if (p.schur) {
    } else if (p.implicit) {
        plan_implicit(p);
        p.ipool = dalloc<float>(p, 24 * n_obs);
        p.rpool = dalloc<float>(p, 2 * n_obs);
        p.lmrec = dalloc<float>(p, LM_REC * (int64_t)n_pt);
        BA_CUDA_TRY(cudaMemsetAsync(p.lmrec, 0, sizeof(float) * LM_REC * (int64_t)n_pt, p.stream));
        require(n_pt < (1 << 30), BA_ERR_INVALID_ARG, "the implicit storage supports fewer than 2^30 landmarks");
        p.pq_part = dalloc<float>(p, 2LL * p.sm_count);
        build_k3_records(p);
        p.tuned = true;  // the tile plans of the stored blocks do not apply
    } else {
        plan_matvec(p);
        p.apool = dalloc<float>(p, p.a_floats);
        p.cpool = dalloc<float>(p, 2 * n_obs + 8);
        p.rot = dalloc<float>(p, 12 * (int64_t)n_pt);
    }
    p.dp2 = dalloc<float>(p, 9 * (int64_t)n_cam);
    p.dl2 = dalloc<float>(p, 3 * (int64_t)n_pt);
    const int64_t nv = 9 * (int64_t)n_cam;
    p.g = dalloc<float>(p, nv);
    p.x = dalloc<float>(p, nv);
    p.r = dalloc<float>(p, nv);
    p.z = dalloc<float>(p, nv);
    p.p = dalloc<float>(p, nv);
    p.q = dalloc<float>(p, nv);
    p.minv = dalloc<float>(p, 81 * (int64_t)n_cam);
    p.mdiag = dalloc<float>(p, 81 * (int64_t)n_cam);
    p.dl = dalloc<float>(p, 3 * (int64_t)n_pt);
    p.partials = dalloc<double>(p, 2LL * p.red_grid + 2);
    BA_CUDA_TRY(cudaMemsetAsync(p.x, 0, sizeof(float) * nv, p.stream));
    BA_CUDA_TRY(cudaMemsetAsync(p.dl, 0, sizeof(float) * 3 * n_pt, p.stream));
    configure_linearize(p);
    if (p.implicit) configure_implicit(p);
    else if (!p.schur) configure_matvec(p);
    sync(p);
}

void set_profiling_impl(Problem& p, int32_t enable) {
    sync(p);
    p.prof.on = false;
    p.prof.pending.clear();
    p.prof.next = 0;
    for (int i = 0; i < PROF_NSLOT; ++i) {
        p.prof.ms[i] = 0.0;
        p.prof.count[i] = 0;
    }
    p.launches = 0;
    p.h2d_bytes = p.d2h_bytes = 0;
    if (enable && p.mv_events.empty()) {
        p.mv_events.resize(2 * PCG_CHUNK);
        for (auto& e : p.mv_events) BA_CUDA_TRY(cudaEventCreate(&e));
    }
    destroy_graph(p);  // recaptured on the next solve, with event nodes only when profiling
    p.prof.on = enable != 0;
}

void get_profile_impl(Problem& p, ba_profile* out) {
    sync(p);
    std::memset(out, 0, sizeof(*out));
    for (int i = 0; i < PROF_NSLOT; ++i) {
        out->ms[i] = p.prof.ms[i];
        out->count[i] = p.prof.count[i];
    }
    out->kernel_launches = p.launches;
    out->h2d_bytes = p.h2d_bytes;
    out->d2h_bytes = p.d2h_bytes;
}

// --- batches of independent problems -----------------------------------------------
thread_local std::string g_batch_create_error;
thread_local std::string g_mlp_create_error;

void create_batch(ba_batch* bh, const ba_problem_desc* descs, int32_t n, const ba_options* opt, void* stream) {
    require(descs != nullptr && n >= 1, BA_ERR_INVALID_ARG, "no problems");
    int64_t tc = 0, tp = 0, to = 0;
    for (int32_t b = 0; b < n; ++b) {
        const ba_problem_desc& d = descs[b];
        require(d.cams && d.pts && d.obs_cam && d.obs_pt && d.obs_xy, BA_ERR_INVALID_ARG, "null input pointer");
        require(d.n_cam >= 1 && d.n_pt >= 1 && d.n_obs >= 2, BA_ERR_INVALID_ARG, "empty problem in the batch");
        for (int64_t o = 0; o < d.n_obs; ++o) {
            require(d.obs_cam[o] >= 0 && d.obs_cam[o] < d.n_cam, BA_ERR_INVALID_ARG,
                    "camera index out of its problem's range");
            require(d.obs_pt[o] >= 0 && d.obs_pt[o] < d.n_pt, BA_ERR_INVALID_ARG,
                    "landmark index out of its problem's range");
        }
        tc += d.n_cam;
        tp += d.n_pt;
        to += d.n_obs;
    }
    require(tc < ((int64_t)1 << 31) && tp < ((int64_t)1 << 31), BA_ERR_INVALID_ARG, "batch too large");
    std::vector<double> cams(9 * tc), pts(3 * tp), xy(2 * to);
    std::vector<int32_t> oc(to), op(to), cam_prob(tc), lm_prob(tp);
    BatchState& B = bh->p.batch;
    B.h_cam_off.assign(n + 1, 0);
    B.h_lm_off.assign(n + 1, 0);
    B.h_obs_off.assign(n + 1, 0);
    for (int32_t b = 0; b < n; ++b) {
        const ba_problem_desc& d = descs[b];
        const int32_t c0 = B.h_cam_off[b], l0 = B.h_lm_off[b];
        const int64_t o0 = B.h_obs_off[b];
        std::memcpy(&cams[9 * (int64_t)c0], d.cams, sizeof(double) * 9 * d.n_cam);
        std::memcpy(&pts[3 * (int64_t)l0], d.pts, sizeof(double) * 3 * d.n_pt);
        std::memcpy(&xy[2 * o0], d.obs_xy, sizeof(double) * 2 * d.n_obs);
        for (int64_t o = 0; o < d.n_obs; ++o) {
            oc[o0 + o] = c0 + d.obs_cam[o];
            op[o0 + o] = l0 + d.obs_pt[o];
        }
        for (int32_t i = 0; i < d.n_cam; ++i) cam_prob[c0 + i] = b;
        for (int32_t i = 0; i < d.n_pt; ++i) lm_prob[l0 + i] = b;
        B.h_cam_off[b + 1] = c0 + d.n_cam;
        B.h_lm_off[b + 1] = l0 + d.n_pt;
        B.h_obs_off[b + 1] = o0 + d.n_obs;
    }
    Problem& p = bh->p;
    create_problem(p, cams.data(), (int32_t)tc, pts.data(), (int32_t)tp, oc.data(), op.data(), xy.data(), to, opt,
                   stream);
    // sorted observations are grouped by landmark and every problem's
    // landmarks are contiguous, so problem b owns sorted positions
    // h_obs_off[b] .. h_obs_off[b + 1] - 1
    B.n_prob = n;
    B.cam_prob = dalloc<int32_t>(p, tc);
    B.lm_prob = dalloc<int32_t>(p, tp);
    B.prob_cam_off = dalloc<int32_t>(p, n + 1);
    B.prob_lm_off = dalloc<int32_t>(p, n + 1);
    B.prob_obs_off = dalloc<int64_t>(p, n + 1);
    B.lam = dalloc<float>(p, n);
    B.pcg = dalloc<PcgScalars>(p, n);
    B.n_done = dalloc<int32_t>(p, 1);
    B.lm = dalloc<BatchLm>(p, n);
    B.cost_a = dalloc<double>(p, n);
    B.cost_b = dalloc<double>(p, n);
    B.n_active = dalloc<int32_t>(p, 1);
    B.n_active_host = static_cast<int32_t*>(pinned_get(sizeof(int32_t)));
    h2d(p, B.cam_prob, cam_prob.data(), tc);
    h2d(p, B.lm_prob, lm_prob.data(), tp);
    h2d(p, B.prob_cam_off, B.h_cam_off.data(), n + 1);
    h2d(p, B.prob_lm_off, B.h_lm_off.data(), n + 1);
    h2d(p, B.prob_obs_off, B.h_obs_off.data(), n + 1);
    bh->init_cams = dalloc<float>(p, 9 * tc);
    bh->init_pts = dalloc<float>(p, 3 * tp);
    BA_CUDA_TRY(cudaMemcpyAsync(bh->init_cams, p.cams, sizeof(float) * 9 * tc, cudaMemcpyDeviceToDevice, p.stream));
    BA_CUDA_TRY(cudaMemcpyAsync(bh->init_pts, p.pts, sizeof(float) * 3 * tp, cudaMemcpyDeviceToDevice, p.stream));
    sync(p);
}

void do_batch_solve(Problem& p, ba_batch_report* reps, ba_batch_summary* sum) {
    BatchState& B = p.batch;
    const int max_it = p.opt.max_lm_iters;
    while ((int)B.iter_events.size() < max_it + 1) {
        cudaEvent_t e;
        BA_CUDA_TRY(cudaEventCreate(&e));
        B.iter_events.push_back(e);
    }
    const int64_t launches0 = p.launches;
    double tune_ms = 0.0;
    BA_CUDA_TRY(cudaEventRecord(B.iter_events[0], p.stream));
    int n_it = 0;
    launch_batch_cost(p, false, B.cost_a);
    launch_batch_start(p);  // lambda0 for every problem
    B.iter_active.assign(1, B.n_prob);
    for (int it = 0; it < max_it; ++it) {
        // K1 for the problems that moved (the first iteration: all; a problem
        // whose last step was rejected keeps its blocks, a stopped one does
        // nothing), then K2 with each problem's damping (undoing the old one
        // where the blocks were kept)
        PhaseTimer tl(p, PROF_LINEARIZE);
        launch_frames(p);
        launch_linearize(p);
        tl.end();
        p.linearized = true;
        PhaseTimer td(p, PROF_DAMP);
        launch_damp(p, false, 1.f);  // per-problem damping from B.lam
        td.end();
        p.damped = true;
        if (p.opt.autotune && !p.tuned) {
            ba_tune_report tr{};
            run_autotune(p, &tr);
            tune_ms = tr.tune_ms;
        }
        do_pcg(p, nullptr);
        PhaseTimer tb(p, PROF_BACKSUB);
        launch_backsub_candidate_cost(p);
        tb.end();
        launch_batch_decide(p, it);
        launch_batch_commit(p);
        BA_CUDA_TRY(cudaEventRecord(B.iter_events[it + 1], p.stream));
        d2h(p, B.n_active_host, B.n_active, 1);
        sync(p);
        n_it = it + 1;
        if (*B.n_active_host == 0) break;
        B.iter_active.push_back(*B.n_active_host);
    }
    B.iter_ms.assign(n_it, 0.f);
    for (int i = 0; i < n_it; ++i)
        BA_CUDA_TRY(cudaEventElapsedTime(&B.iter_ms[i], B.iter_events[i], B.iter_events[i + 1]));
    p.linearized = p.damped = p.solved = p.backsubbed = false;
    std::vector<BatchLm> lm(B.n_prob);
    d2h(p, lm.data(), B.lm, B.n_prob);
    sync(p);
    std::vector<double> t_end(n_it + 1, 0.0);
    for (int i = 1; i <= n_it; ++i) {
        float ms = 0.f;
        BA_CUDA_TRY(cudaEventElapsedTime(&ms, B.iter_events[0], B.iter_events[i]));
        t_end[i] = ms;
    }
    if (reps) {
        for (int b = 0; b < B.n_prob; ++b) {
            ba_batch_report& r = reps[b];
            r.iterations = lm[b].iter;
            r.accepted = lm[b].accepted;
            r.cg_iters = lm[b].cg_total;
            r.stop = lm[b].stop;
            r.initial_cost = lm[b].cost0;
            r.final_cost = lm[b].cost;
            r.lambda = lm[b].lambda;
            const int f = lm[b].finish >= 0 ? lm[b].finish + 1 : n_it;
            r.solve_ms = t_end[std::min(f, n_it)];
        }
    }
    if (sum) {
        sum->n_problems = B.n_prob;
        sum->lm_iterations = n_it;
        sum->tuned_ksmall = p.mv_plan.ksmall;
        sum->tuned_small_bytes = p.mv_plan.small_bytes;
        sum->total_ms = t_end[n_it];
        sum->tune_ms = tune_ms;
        sum->kernel_launches = p.launches - launches0;
    }
}

// Synchronises the model's stream and reads its error word: a tensor-core
// wait that gave up fails the call with BA_ERR_TIMEOUT (the word is cleared).
void mlp_sync_checked(Mlp& m) {
    uint32_t e = 0;
    BA_CUDA_TRY(cudaMemcpyAsync(&e, m.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, m.stream));
    BA_CUDA_TRY(cudaStreamSynchronize(m.stream));
    if (e) {
        BA_CUDA_TRY(cudaMemsetAsync(m.err, 0, sizeof(uint32_t), m.stream));
        if (e & ERRBIT_TIMEOUT)
            throw Error{BA_ERR_TIMEOUT, "a bounded tensor-core wait of the model gave up; outputs are invalid"};
    }
}

}  // namespace

namespace sqrtba {
// failure text of calls without a handle, read back by ba_last_error(NULL)
void set_create_error(const std::string& m) { g_create_error = m; }
}  // namespace sqrtba

extern "C" {

void ba_default_options(ba_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->lambda0 = 1e-4;
    o->max_lm_iters = 50;
    o->func_tol = 1e-6;
    o->max_cg_iters = 500;
    o->cg_eta = 0.1;
    o->use_graph = 1;
}

ba_status ba_create(const double* cams, int32_t n_cam, const double* pts, int32_t n_pt, const int32_t* obs_cam,
                    const int32_t* obs_pt, const double* obs_xy, int64_t n_obs, const ba_options* opt,
                    void* cuda_stream, ba_problem** out) {
    ba_problem* h = nullptr;
    g_create_error.clear();
    try {
        require(out != nullptr, BA_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        h = new ba_problem();
        create_problem(h->p, cams, n_cam, pts, n_pt, obs_cam, obs_pt, obs_xy, n_obs, opt, cuda_stream);
        *out = h;
        return BA_OK;
    } catch (const Error& e) {
        g_create_error = e.msg;
        if (h) {
            free_all(h->p);
            delete h;
        }
        return e.code;
    } catch (const std::bad_alloc&) {
        g_create_error = "host allocation failed";
        if (h) {
            free_all(h->p);
            delete h;
        }
        return BA_ERR_OOM;
    }
}

ba_status ba_destroy(ba_problem* h) {
    if (!h) return BA_OK;
    if (h->p.stream) cudaStreamSynchronize(h->p.stream);
    free_all(h->p);
    delete h;
    return BA_OK;
}

ba_status ba_linearize(ba_problem* h) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    do_linearize(h->p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_linearize_damped(ba_problem* h, double lambda) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    require(std::isfinite(lambda) && lambda > 0.0, BA_ERR_INVALID_ARG, "lambda must be positive and finite");
    do_linearize(h->p, true, lambda);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_marginalize_qr(ba_problem* h, double lambda) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    do_marginalize(h->p, lambda);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_pcg_solve(ba_problem* h, ba_pcg_report* rep) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    do_pcg(h->p, rep);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_backsubstitute(ba_problem* h, double* model_cost) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    const double m = do_backsub(h->p);
    if (model_cost) *model_cost = m;
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_eval_cost(ba_problem* h, int32_t candidate, double* cost) {
    if (!h || !cost) return BA_ERR_INVALID_ARG;
    API_TRY
    *cost = do_eval_cost(h->p, candidate != 0);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_lm_step(ba_problem* h, ba_lm_report* rep) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    do_lm_step(h->p, rep);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_solve(ba_problem* h, ba_lm_report* reps, int32_t max_reports, int32_t* n_reports) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    int32_t n = 0;
    while (!h->p.stopped) {
        ba_lm_report r;
        do_lm_step(h->p, &r);
        if (reps && n < max_reports) reps[n] = r;
        ++n;
    }
    if (n_reports) *n_reports = n;
    return BA_OK;
    API_CATCH(h)
}

// A process-wide page-locked staging buffer for reading the state back
// (grow-only; one caller at a time): the device-to-host copy then runs at the
// link's speed instead of through the driver's pageable bounce buffers, and a
// problem created per solve does not pay for page-locking each time.
struct HostStage {
    std::mutex mu;
    void* ptr = nullptr;
    size_t bytes = 0;
};
HostStage& host_stage() {
    static HostStage s;
    return s;
}

ba_status ba_get_params(ba_problem* h, double* cams, double* pts) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    const size_t nc = 9 * (size_t)p.n_cam, nx = 3 * (size_t)p.n_pt;
    HostStage& hs = host_stage();
    std::lock_guard<std::mutex> lock(hs.mu);
    const size_t need = sizeof(float) * (nc + nx);
    if (hs.bytes < need) {
        if (hs.ptr) cudaFreeHost(hs.ptr);
        hs.ptr = nullptr;
        hs.bytes = 0;
        BA_CUDA_TRY(cudaMallocHost(&hs.ptr, need));
        hs.bytes = need;
    }
    float* c = static_cast<float*>(hs.ptr);
    float* x = c + nc;
    if (cams) d2h(p, c, p.cams, (int64_t)nc);
    if (pts) d2h(p, x, p.pts, (int64_t)nx);
    sync(p);
    if (cams)
        for (size_t i = 0; i < nc; ++i) cams[i] = c[i];
    if (pts)
        for (size_t i = 0; i < nx; ++i) pts[i] = x[i];
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_set_params(ba_problem* h, const double* cams, const double* pts) {
    if (!h || !cams || !pts) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    std::vector<float> c(9 * (size_t)p.n_cam), x(3 * (size_t)p.n_pt);
    for (size_t i = 0; i < c.size(); ++i) {
        require(std::isfinite(cams[i]), BA_ERR_INVALID_ARG, "non-finite camera value");
        c[i] = (float)cams[i];
    }
    for (size_t i = 0; i < x.size(); ++i) {
        require(std::isfinite(pts[i]), BA_ERR_INVALID_ARG, "non-finite point value");
        x[i] = (float)pts[i];
    }
    h2d(p, p.cams, c.data(), (int64_t)c.size());
    h2d(p, p.pts, x.data(), (int64_t)x.size());
    sync(p);
    p.linearized = p.damped = p.solved = p.backsubbed = false;
    p.cost_valid = p.cost_pending = false;
    p.lambda = p.opt.lambda0;
    p.nu = 2.0;
    p.iteration = 0;
    p.stopped = false;
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_set_options(ba_problem* h, const ba_options* opt) {
    if (!h || !opt) return BA_ERR_INVALID_ARG;
    API_TRY
    require(opt->lambda0 > 0 && opt->max_lm_iters >= 1 && opt->max_cg_iters >= 1 && opt->cg_eta > 0 &&
            (opt->pipeline_stages == 0 || (opt->pipeline_stages >= 4 && opt->pipeline_stages <= 6)) &&
            std::isfinite(opt->huber_delta) && opt->huber_delta >= 0.0,
            BA_ERR_INVALID_ARG, "invalid options");
    Problem& p = h->p;
    require(opt->implicit_blocks == p.opt.implicit_blocks && opt->schur_explicit == p.opt.schur_explicit,
            BA_ERR_INVALID_ARG, "implicit_blocks and schur_explicit are fixed when the problem is created");
    sync(p);
    const bool graph_change = opt->use_graph != p.opt.use_graph || opt->pipeline_stages != p.opt.pipeline_stages;
    if (opt->huber_delta != p.opt.huber_delta) {
        // another cost function: the energy and the linearisation are recomputed
        p.cost_valid = false;
        p.linearized = p.damped = p.solved = p.backsubbed = false;
    }
    p.opt = *opt;
    if (graph_change) destroy_graph(p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_get_state(ba_problem* h, ba_lm_state* s) {
    if (!h || !s) return BA_ERR_INVALID_ARG;
    s->lambda = h->p.lambda;
    s->nu = h->p.nu;
    s->iteration = h->p.iteration;
    s->stopped = h->p.stopped ? 1 : 0;
    return BA_OK;
}

ba_status ba_set_state(ba_problem* h, const ba_lm_state* s) {
    if (!h || !s) return BA_ERR_INVALID_ARG;
    if (!(s->lambda > 0) || !(s->nu >= 1) || s->iteration < 0) {
        set_error(h, "invalid LM state");
        return BA_ERR_INVALID_ARG;
    }
    h->p.lambda = s->lambda;
    h->p.nu = s->nu;
    h->p.iteration = s->iteration;
    h->p.stopped = s->stopped != 0;
    return BA_OK;
}

ba_status ba_get_info(ba_problem* h, ba_info* info) {
    if (!h || !info) return BA_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_cam = h->p.n_cam;
    info->n_pt = h->p.n_pt;
    info->n_obs = h->p.n_obs;
    info->a_pool_floats = h->p.a_floats;
    info->sum_k2 = h->p.sum_k2;
    info->k_max = h->p.k_max;
    info->device_bytes = h->p.device_bytes;
    return BA_OK;
}

ba_status ba_set_profiling(ba_problem* h, int32_t enable) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    set_profiling_impl(h->p, enable);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_get_profile(ba_problem* h, ba_profile* out) {
    if (!h || !out) return BA_ERR_INVALID_ARG;
    API_TRY
    get_profile_impl(h->p, out);
    return BA_OK;
    API_CATCH(h)
}

const char* ba_last_error(const ba_problem* h) {
    return h ? h->p.last_error.c_str() : g_create_error.c_str();
}

// --- inspection exports ---------------------------------------------------------
ba_status ba_debug_export_order(ba_problem* h, int32_t* perm, int64_t* pt_off, int64_t* cam_off,
                                int32_t* cam_list) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    std::vector<int32_t> po(p.n_pt + 1), co(p.n_cam + 1);
    if (perm) d2h(p, perm, p.perm, p.n_obs);
    if (cam_list) d2h(p, cam_list, p.cam_list, p.n_obs);
    d2h(p, po.data(), p.pt_off, p.n_pt + 1);
    d2h(p, co.data(), p.cam_off, p.n_cam + 1);
    sync(p);
    if (pt_off)
        for (int i = 0; i <= p.n_pt; ++i) pt_off[i] = po[i];
    if (cam_off)
        for (int i = 0; i <= p.n_cam; ++i) cam_off[i] = co[i];
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_debug_export_landmark(ba_problem* h, int32_t j, int32_t k_cap, float* top, float* a, float* c,
                                   float* rot, int32_t* k_out) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    require(j >= 0 && j < p.n_pt, BA_ERR_INVALID_ARG, "landmark index out of range");
    require(p.linearized, BA_ERR_STATE, "not linearised");
    int32_t off[2], coff = 0;
    int64_t aoff = 0;
    d2h(p, off, p.pt_off + j, 2);
    d2h(p, &aoff, p.a_off + j, 1);
    d2h(p, &coff, p.c_off + j, 1);
    sync(p);
    const int k = off[1] - off[0];
    if (k_out) *k_out = k;
    require(k <= k_cap, BA_ERR_INVALID_ARG, "k exceeds k_cap");
    require(!p.implicit || (!a && !c && !rot), BA_ERR_INVALID_ARG,
            "implicit storage: only the (undamped) top rows can be exported");
    require(!p.schur, BA_ERR_INVALID_ARG, "the explicit Schur complement stores no landmark blocks");
    const int64_t ncol = 9 * (int64_t)k;
    if (top && p.implicit) {  // rebuilt from the records (the implicit storage keeps no top rows)
        float* d_top = nullptr;
        BA_CUDA_TRY(cudaMalloc(&d_top, sizeof(float) * 3 * (ncol + 4)));
        std::unique_ptr<float, decltype(&cudaFree)> hold(d_top, &cudaFree);
        launch_implicit_top_rows(p, j, k, d_top);
        d2h(p, top, d_top, 3 * (ncol + 4));
        sync(p);
    } else if (top) {
        d2h(p, top, p.tpool + top_offset(off[0], j), 3 * (ncol + 4));
    }
    if (a) d2h(p, a, p.apool + aoff, 2 * (int64_t)k * ncol);
    if (c) d2h(p, c, p.cpool + coff, 2 * (int64_t)k);
    if (rot) d2h(p, rot, p.rot + 12 * (int64_t)j, 12);
    sync(p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_debug_export_damping(ba_problem* h, float* dp2, float* dl2) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    if (dp2) d2h(p, dp2, p.dp2, 9 * (int64_t)p.n_cam);
    if (dl2) d2h(p, dl2, p.dl2, 3 * (int64_t)p.n_pt);
    sync(p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_debug_export_jacobians(ba_problem* h, float* r, float* jp, float* jl) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    float *dr = nullptr, *djp = nullptr, *djl = nullptr;
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&dr, sizeof(float) * 2 * p.n_obs, device_pool(), p.stream));
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&djp, sizeof(float) * 18 * p.n_obs, device_pool(), p.stream));
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&djl, sizeof(float) * 6 * p.n_obs, device_pool(), p.stream));
    launch_export_jacobians(p, dr, djp, djl);
    if (r) d2h(p, r, dr, 2 * p.n_obs);
    if (jp) d2h(p, jp, djp, 18 * p.n_obs);
    if (jl) d2h(p, jl, djl, 6 * p.n_obs);
    cudaFreeAsync(dr, p.stream);
    cudaFreeAsync(djp, p.stream);
    cudaFreeAsync(djl, p.stream);
    sync(p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_debug_export_rcs_diag(ba_problem* h, float* m, float* g) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    require(p.solved, BA_ERR_STATE, "no PCG solve yet");
    if (m) d2h(p, m, p.mdiag, 81 * (int64_t)p.n_cam);
    if (g) d2h(p, g, p.g, 9 * (int64_t)p.n_cam);
    sync(p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_debug_matvec(ba_problem* h, const float* v, float* y) {
    if (!h || !v || !y) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    require(p.damped, BA_ERR_STATE, "blocks are not marginalised");
    const int64_t n = 9 * (int64_t)p.n_cam;
    float *dv = nullptr, *dy = nullptr;
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&dv, sizeof(float) * n, device_pool(), p.stream));
    BA_CUDA_TRY(cudaMallocFromPoolAsync(&dy, sizeof(float) * n, device_pool(), p.stream));
    h2d(p, dv, v, n);
    launch_matvec(p, dv, dy, true);
    d2h(p, y, dy, n);
    cudaFreeAsync(dv, p.stream);
    cudaFreeAsync(dy, p.stream);
    sync_checked(p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_debug_fail_matvec(ba_problem* h, int32_t tile, double wait_ms) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    if (tile >= 0) {
        require(wait_ms > 0.0 && wait_ms <= 2000.0, BA_ERR_INVALID_ARG, "wait_ms must be in (0, 2000]");
        p.dbg_fail_tile = tile;
        p.dbg_wait_ns = (uint64_t)(wait_ms * 1e6);
    } else {
        p.dbg_fail_tile = -1;
        p.dbg_wait_ns = 0;
    }
    destroy_graph(p);  // the captured launches hold the old arguments
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_debug_export_step(ba_problem* h, float* dp, float* dl) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    Problem& p = h->p;
    if (dp) d2h(p, dp, p.x, 9 * (int64_t)p.n_cam);
    if (dl) d2h(p, dl, p.dl, 3 * (int64_t)p.n_pt);
    sync(p);
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_autotune(ba_problem* h, ba_tune_report* rep) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    run_autotune(h->p, rep);
    return BA_OK;
    API_CATCH(h)
}

// --- batches -----------------------------------------------------------------------
#define BATCH_TRY try {
#define BATCH_CATCH(b)                                \
    }                                                 \
    catch (const Error& e) {                          \
        (b)->p.last_error = e.msg;                    \
        return e.code;                                \
    }                                                 \
    catch (const std::bad_alloc&) {                   \
        (b)->p.last_error = "host allocation failed"; \
        return BA_ERR_OOM;                            \
    }                                                 \
    catch (...) {                                     \
        (b)->p.last_error = "unexpected exception";   \
        return BA_ERR_CUDA;                           \
    }

ba_status ba_batch_create(const ba_problem_desc* descs, int32_t n, const ba_options* opt, void* cuda_stream,
                          ba_batch** out) {
    ba_batch* b = nullptr;
    g_batch_create_error.clear();
    try {
        require(out != nullptr, BA_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        b = new ba_batch();
        create_batch(b, descs, n, opt, cuda_stream);
        *out = b;
        return BA_OK;
    } catch (const Error& e) {
        g_batch_create_error = e.msg;
        if (b) {
            free_all(b->p);
            delete b;
        }
        return e.code;
    } catch (const std::bad_alloc&) {
        g_batch_create_error = "host allocation failed";
        if (b) {
            free_all(b->p);
            delete b;
        }
        return BA_ERR_OOM;
    }
}

ba_status ba_batch_destroy(ba_batch* b) {
    if (!b) return BA_OK;
    if (b->p.stream) cudaStreamSynchronize(b->p.stream);
    free_all(b->p);
    delete b;
    return BA_OK;
}

ba_status ba_batch_solve(ba_batch* b, ba_batch_report* reports, ba_batch_summary* summary) {
    if (!b) return BA_ERR_INVALID_ARG;
    BATCH_TRY
    do_batch_solve(b->p, reports, summary);
    return BA_OK;
    BATCH_CATCH(b)
}

ba_status ba_batch_restart(ba_batch* b) {
    if (!b) return BA_ERR_INVALID_ARG;
    BATCH_TRY
    Problem& p = b->p;
    BA_CUDA_TRY(cudaMemcpyAsync(p.cams, b->init_cams, sizeof(float) * 9 * p.n_cam, cudaMemcpyDeviceToDevice,
                                p.stream));
    BA_CUDA_TRY(cudaMemcpyAsync(p.pts, b->init_pts, sizeof(float) * 3 * p.n_pt, cudaMemcpyDeviceToDevice,
                                p.stream));
    p.linearized = p.damped = p.solved = p.backsubbed = false;
    return BA_OK;
    BATCH_CATCH(b)
}

ba_status ba_batch_get_params(ba_batch* b, int32_t i, double* cams, double* pts) {
    if (!b) return BA_ERR_INVALID_ARG;
    BATCH_TRY
    Problem& p = b->p;
    const BatchState& B = p.batch;
    require(i >= 0 && i < B.n_prob, BA_ERR_INVALID_ARG, "problem index out of range");
    const int32_t c0 = B.h_cam_off[i], nc = B.h_cam_off[i + 1] - c0;
    const int32_t l0 = B.h_lm_off[i], nl = B.h_lm_off[i + 1] - l0;
    std::vector<float> c(9 * (size_t)nc), x(3 * (size_t)nl);
    if (cams) d2h(p, c.data(), p.cams + 9 * (int64_t)c0, (int64_t)c.size());
    if (pts) d2h(p, x.data(), p.pts + 3 * (int64_t)l0, (int64_t)x.size());
    sync(p);
    if (cams)
        for (size_t k = 0; k < c.size(); ++k) cams[k] = c[k];
    if (pts)
        for (size_t k = 0; k < x.size(); ++k) pts[k] = x[k];
    return BA_OK;
    BATCH_CATCH(b)
}

ba_status ba_batch_set_profiling(ba_batch* b, int32_t enable) {
    if (!b) return BA_ERR_INVALID_ARG;
    BATCH_TRY
    set_profiling_impl(b->p, enable);
    return BA_OK;
    BATCH_CATCH(b)
}

ba_status ba_batch_get_profile(ba_batch* b, ba_profile* out) {
    if (!b || !out) return BA_ERR_INVALID_ARG;
    BATCH_TRY
    get_profile_impl(b->p, out);
    return BA_OK;
    BATCH_CATCH(b)
}

ba_status ba_batch_iterations(ba_batch* b, int32_t cap, int32_t* active, float* ms, int32_t* n) {
    if (!b || !n || cap < 0) return BA_ERR_INVALID_ARG;
    const BatchState& B = b->p.batch;
    const int m = (int)B.iter_ms.size();
    *n = m;
    for (int i = 0; i < std::min(m, (int)cap); ++i) {
        if (active) active[i] = i < (int)B.iter_active.size() ? B.iter_active[i] : 0;
        if (ms) ms[i] = B.iter_ms[i];
    }
    return BA_OK;
}

ba_status ba_batch_get_info(ba_batch* b, ba_info* info) {
    if (!b || !info) return BA_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_cam = b->p.n_cam;
    info->n_pt = b->p.n_pt;
    info->n_obs = b->p.n_obs;
    info->a_pool_floats = b->p.a_floats;
    info->sum_k2 = b->p.sum_k2;
    info->k_max = b->p.k_max;
    info->device_bytes = b->p.device_bytes;
    return BA_OK;
}

const char* ba_batch_last_error(const ba_batch* b) {
    return b ? b->p.last_error.c_str() : g_batch_create_error.c_str();
}

// --- learned warm start / preconditioner correction -----------------------------
#define MLP_TRY try {
#define MLP_CATCH(h)                                  \
    }                                                 \
    catch (const Error& e) {                          \
        (h)->m.last_error = e.msg;                    \
        return e.code;                                \
    }                                                 \
    catch (const std::bad_alloc&) {                   \
        (h)->m.last_error = "host allocation failed"; \
        return BA_ERR_OOM;                            \
    }

ba_status ba_mlp_create(const float* params, void* cuda_stream, ba_mlp** out) {
    ba_mlp* h = nullptr;
    g_mlp_create_error.clear();
    try {
        require(out != nullptr && params != nullptr, BA_ERR_INVALID_ARG, "null pointer");
        *out = nullptr;
        for (int64_t i = 0; i < ML_P; ++i) require(std::isfinite(params[i]), BA_ERR_INVALID_ARG, "non-finite parameter");
        h = new ba_mlp();
        mlp_init(h->m, params, (cudaStream_t)cuda_stream);
        *out = h;
        return BA_OK;
    } catch (const Error& e) {
        g_mlp_create_error = e.msg;
        if (h) {
            mlp_free(h->m);
            delete h;
        }
        return e.code;
    } catch (const std::bad_alloc&) {
        g_mlp_create_error = "host allocation failed";
        if (h) {
            mlp_free(h->m);
            delete h;
        }
        return BA_ERR_OOM;
    }
}

ba_status ba_mlp_destroy(ba_mlp* h) {
    if (!h) return BA_OK;
    mlp_free(h->m);
    delete h;
    return BA_OK;
}

ba_status ba_mlp_get_params(ba_mlp* h, float* params) {
    if (!h || !params) return BA_ERR_INVALID_ARG;
    MLP_TRY
    BA_CUDA_TRY(cudaMemcpyAsync(params, h->m.master, sizeof(float) * ML_P, cudaMemcpyDeviceToHost, h->m.stream));
    BA_CUDA_TRY(cudaStreamSynchronize(h->m.stream));
    return BA_OK;
    MLP_CATCH(h)
}

ba_status ba_mlp_forward(ba_mlp* h, const float* d_feats, int32_t n, float* d_out) {
    if (!h || !d_feats || !d_out || n < 1) return BA_ERR_INVALID_ARG;
    MLP_TRY
    mlp_forward(h->m, d_feats, n, d_out);
    mlp_sync_checked(h->m);
    return BA_OK;
    MLP_CATCH(h)
}

ba_status ba_mlp_prepare(ba_mlp* h, const float* d_M, const float* d_g, const float* d_xstar, const int32_t* d_count,
                         int32_t n, float* d_feats, float* d_aux) {
    if (!h || !d_M || !d_g || !d_count || !d_feats || !d_aux || n < 1) return BA_ERR_INVALID_ARG;
    MLP_TRY
    mlp_prepare(h->m.stream, d_M, d_g, d_xstar, d_count, n, d_feats, d_aux);
    BA_CUDA_TRY(cudaStreamSynchronize(h->m.stream));
    return BA_OK;
    MLP_CATCH(h)
}

ba_status ba_mlp_loss_grad(ba_mlp* h, const float* d_feats, const float* d_aux, int32_t n, double* loss,
                           float* grads) {
    if (!h || !d_feats || !d_aux || n < 1) return BA_ERR_INVALID_ARG;
    MLP_TRY
    const double l = mlp_loss_grad(h->m, d_feats, d_aux, n);
    if (loss) *loss = l;
    if (grads)
        BA_CUDA_TRY(cudaMemcpyAsync(grads, h->m.grad, sizeof(float) * ML_P, cudaMemcpyDeviceToHost, h->m.stream));
    mlp_sync_checked(h->m);
    return BA_OK;
    MLP_CATCH(h)
}

ba_status ba_mlp_train_step(ba_mlp* h, const float* d_feats, const float* d_aux, int32_t n, float lr,
                            double* loss) {
    if (!h || !d_feats || !d_aux || n < 1 || !(lr > 0.f)) return BA_ERR_INVALID_ARG;
    MLP_TRY
    const double l = mlp_loss_grad(h->m, d_feats, d_aux, n);
    mlp_adam(h->m, lr, 0.9f, 0.999f, 1e-8f);
    if (loss) *loss = l;
    return BA_OK;
    MLP_CATCH(h)
}

const char* ba_mlp_last_error(const ba_mlp* h) { return h ? h->m.last_error.c_str() : g_mlp_create_error.c_str(); }

ba_status ba_set_learned(ba_problem* h, ba_mlp* model) {
    if (!h) return BA_ERR_INVALID_ARG;
    API_TRY
    sync(h->p);
    h->p.mlp = model ? &model->m : nullptr;
    return BA_OK;
    API_CATCH(h)
}

ba_status ba_learned_fallbacks(ba_problem* h, int64_t* count) {
    if (!h || !count) return BA_ERR_INVALID_ARG;
    *count = h->p.learned_fallbacks;
    return BA_OK;
}

}  // extern "C"
