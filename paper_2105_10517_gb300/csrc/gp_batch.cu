// gp_batch.cu -- many GP solves served together: admission by device-memory
// footprint, one launch per substep (and solve kind) for all running instances
// of a precision (one CTA per work item, or persistent),
// convergence checks between ticks, retirement that frees memory for the next
// admission (continuous batching).  Each instance keeps its psi, intermediate
// and Thomas coefficient tables resident on the device for its whole life.
//
// An instance's arithmetic is the same alone and in any mix: batched CTAs run
// the single-instance kernel bodies with the instance's own tiling and thread
// count, and its normalisation sums the same partials in the same order.
#include "gp_handle.cuh"

#include <algorithm>
#include <cmath>
#include <deque>
#include <map>
#include <new>
#include <vector>

using namespace gpspin;

namespace {

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;
    int reserve(size_t n)
    {
        if (n <= cap) return GP_OK;
        cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t c = std::max<size_t>(n, 64);
        if (!dalloc(&p, c * sizeof(T))) return GP_ERR_OOM;
        cap = c;
        return GP_OK;
    }
    void release()
    {
        cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

struct Request {
    long long id = 0;
    gp_params p{};
    gp_request r{};
    int state = GP_REQ_QUEUED;
    gp_handle* h = nullptr;
    size_t bytes = 0;
    long long steps = 0;
    bool have_e = false;
    double e_last = 0;
    gp_obs obs{};
    int error = GP_OK;        // status that failed the request
    std::vector<double> psi;  // result, complex128, after completion
};

// Work items of one pass whose tilings share a solve kind: the shared-memory
// solve (class 0) or the register-resident solve of chunk length 16, 24, 32.
constexpr int kSolveClasses = 4;
constexpr int kClassM[kSolveClasses] = {0, 16, 24, 32};

int solve_class(const LineTiling& t)
{
    if (!t.single) return 0;
    return t.m == 16 ? 1 : (t.m == 24 ? 2 : 3);
}

struct PassList {
    std::vector<int2> items;
    int threads = 0;
    size_t smem = 0;
    DevBuf<int2> d;
    void clear()
    {
        items.clear();
        threads = 0;
        smem = 0;
    }
    void add(int inst, const LineTiling& t)
    {
        const int n = y_blocks(t);
        for (int c = 0; c < n; ++c) items.push_back(make_int2(inst, c));
        threads = std::max(threads, t.threads);
        smem = std::max(smem, t.smem);
    }
};

// Counts (device) per group: work items of the x and y classes, then instances.
constexpr int kGroupCounts = 2 * kSolveClasses + 1;

template <typename C>
struct Group {
    std::vector<PassArgsT<C>> ax, ay;
    PassList lx[kSolveClasses], ly[kSolveClasses];
    std::vector<FinArgs> fin;
    DevBuf<PassArgsT<C>> dax, day;
    DevBuf<FinArgs> dfin;
    // CUDA graph of one tick's launches and the launch lists it was captured for:
    // replayed while the running set (and so every argument) is unchanged
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> sig;
    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        sig.clear();
    }
    // bytes of everything the tick's launches read: pass and finalize arguments,
    // work lists, steps per tick
    std::vector<unsigned char> signature(int steps) const
    {
        std::vector<unsigned char> v;
        auto put = [&v](const void* p, size_t n) {
            const unsigned char* c = static_cast<const unsigned char*>(p);
            v.insert(v.end(), c, c + n);
        };
        put(&steps, sizeof steps);
        put(ax.data(), ax.size() * sizeof(ax[0]));
        put(ay.data(), ay.size() * sizeof(ay[0]));
        put(fin.data(), fin.size() * sizeof(fin[0]));
        for (int c = 0; c < kSolveClasses; ++c) {
            const size_t nx = lx[c].items.size(), ny = ly[c].items.size();
            put(&nx, sizeof nx);
            put(lx[c].items.data(), nx * sizeof(int2));
            put(&ny, sizeof ny);
            put(ly[c].items.data(), ny * sizeof(int2));
        }
        return v;
    }
    void clear()
    {
        ax.clear();
        ay.clear();
        for (int c = 0; c < kSolveClasses; ++c) {
            lx[c].clear();
            ly[c].clear();
        }
        fin.clear();
    }
    void release()
    {
        drop_graph();
        dax.release();
        day.release();
        for (int c = 0; c < kSolveClasses; ++c) {
            lx[c].d.release();
            ly[c].d.release();
        }
        dfin.release();
    }
};

}  // namespace

struct gp_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t max_bytes = 0, used_bytes = 0;
    int check_every = 100;
    long long next_id = 1;
    std::deque<long long> queue;
    std::map<long long, Request> reqs;
    Group<double2> g64;
    Group<float2> g32;
    int* counts = nullptr;  // device: kGroupCounts per precision group (complex128, complex64)
    int* work = nullptr;    // device: the persistent launches' item counters, two ints per group
    // batched launch form: < 0 one CTA per item (the default: measured 1-6% faster
    // than the persistent form on the serving mix); 0 persistent, one CTA per
    // resident slot; > 0 persistent with at most that many CTAs
    int persist = -1;
    int* flag = nullptr;
    int max_queued = 0;     // 0: no limit on queued requests
    long long max_sites = 0;  // 0: no limit on the grid points of the running solves
    bool graphs = true;     // replay captured ticks while the running set is unchanged
    cudaStream_t stream32 = nullptr;  // the complex64 group runs beside the complex128 one
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

#define BK(x)                                                  \
    do {                                                       \
        if (report_cuda((x), #x) != 0) return GP_ERR_CUDA;     \
    } while (0)

int policy_precision(int policy) { return policy == GP_POLICY_FP32_REFINE ? GP_FP32_MIXED : GP_FP64; }

LineTiling with_bulk(LineTiling t, int bulk)
{
    t.bulk = bulk;
    return t;
}

// Puts one running instance into its precision group's launch lists.
template <typename C>
void add_instance(Group<C>& g, gp_handle* h, const PassArgsT<C>& ax, PassArgsT<C> ay)
{
    const int inst = (int)g.ax.size();
    ay.partials = h->partials;
    g.ax.push_back(ax);
    g.ay.push_back(ay);
    g.lx[solve_class(ax.t)].add(inst, ax.t);
    g.ly[solve_class(ay.t)].add(inst, ay.t);
    g.fin.push_back(FinArgs{h->partials, y_blocks(ay.t), cell(h), h->scal});
}

// The launches of `steps` steps of one group: per step the x-passes of every
// solve kind, the y-passes, then the normalisation of every instance.  The
// launches of a group run in order on one stream, so a persistent launch's
// counters (work) are free again when the next one starts.
template <typename C>
int enqueue_group(gp_batch* b, Group<C>& g, int* counts, int* work, int steps, cudaStream_t s)
{
    const int n_inst = (int)g.fin.size();
    int* w = b->persist >= 0 ? work : nullptr;
    const int cap = std::max(0, b->persist);
    for (int k = 0; k < steps; ++k) {
        for (int c = 0; c < kSolveClasses; ++c) {
            const PassList& l = g.lx[c];
            if (!l.items.empty() && launch_xpass_batched(g.dax.p, l.d.p, counts + c, (int)l.items.size(), l.threads,
                                                         l.smem, GP_IMAG, s, kClassM[c], w, cap))
                return GP_ERR_CUDA;
        }
        for (int c = 0; c < kSolveClasses; ++c) {
            const PassList& l = g.ly[c];
            if (!l.items.empty() && launch_ypass_batched(g.day.p, l.d.p, counts + kSolveClasses + c,
                                                         (int)l.items.size(), l.threads, l.smem, GP_IMAG, s,
                                                         kClassM[c], w, cap))
                return GP_ERR_CUDA;
        }
        if (launch_finalize_norm_batched(g.dfin.p, counts + 2 * kSolveClasses, n_inst, b->flag, s)) return GP_ERR_CUDA;
    }
    return GP_OK;
}

// One tick of a group on stream s.  While the running set is unchanged the tick
// replays the CUDA graph captured for it; after a change the launch lists are
// uploaded, the tick runs directly and is captured for the next ticks.
template <typename C>
int upload_and_run(gp_batch* b, Group<C>& g, int* counts, int* work, int steps, cudaStream_t s)
{
    if (g.ax.empty()) {
        g.drop_graph();
        return GP_OK;
    }
    std::vector<unsigned char> sig;
    if (b->graphs) {
        sig = g.signature(steps);
        if (g.exec && sig == g.sig) {
            BK(cudaGraphLaunch(g.exec, s));
            return GP_OK;
        }
    }
    g.drop_graph();
    int st;
    if ((st = g.dax.reserve(g.ax.size())) || (st = g.day.reserve(g.ay.size())) || (st = g.dfin.reserve(g.fin.size())))
        return st;
    int n[kGroupCounts];
    for (int c = 0; c < kSolveClasses; ++c) {
        PassList* lists[2] = {&g.lx[c], &g.ly[c]};
        for (int d = 0; d < 2; ++d) {
            PassList& l = *lists[d];
            n[d * kSolveClasses + c] = (int)l.items.size();
            if (l.items.empty()) continue;
            if ((st = l.d.reserve(l.items.size()))) return st;
            BK(cudaMemcpyAsync(l.d.p, l.items.data(), l.items.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        }
    }
    n[2 * kSolveClasses] = (int)g.fin.size();
    BK(cudaMemcpyAsync(g.dax.p, g.ax.data(), g.ax.size() * sizeof(g.ax[0]), cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(g.day.p, g.ay.data(), g.ay.size() * sizeof(g.ay[0]), cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(g.dfin.p, g.fin.data(), g.fin.size() * sizeof(FinArgs), cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(counts, n, sizeof(n), cudaMemcpyHostToDevice, s));
    // the direct launches also set the kernels' shared-memory attributes, which
    // the captured launches then find in place
    if ((st = enqueue_group(b, g, counts, work, steps, s))) return st;
    if (b->graphs) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int cst = enqueue_group(b, g, counts, work, steps, s);
            const cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (cst == GP_OK && e == cudaSuccess && graph && cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess)
                g.sig.swap(sig);
            else
                g.exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();  // a failed capture only means direct launches next tick
    }
    return GP_OK;
}

void retire(gp_batch* b, Request& q, int state)
{
    if (q.h) {
        q.psi.resize(2 * n_elems(q.h));
        if (gp_get_state(q.h, q.psi.data()) != GP_OK) {
            q.psi.clear();
            state = GP_REQ_FAILED;
        }
        gp_destroy(q.h);
        q.h = nullptr;
        b->used_bytes -= q.bytes;
    }
    q.state = state;
}

int running_count(const gp_batch* b)
{
    int n = 0;
    for (const auto& kv : b->reqs) n += kv.second.state == GP_REQ_RUNNING;
    return n;
}

long long running_sites(const gp_batch* b)
{
    long long n = 0;
    for (const auto& kv : b->reqs)
        if (kv.second.state == GP_REQ_RUNNING) n += (long long)kv.second.p.nx * kv.second.p.ny;
    return n;
}

// Admits queued requests in arrival order while their footprint fits.
int admit(gp_batch* b)
{
    while (!b->queue.empty()) {
        Request& q = b->reqs[b->queue.front()];
        if (q.bytes > b->max_bytes) {  // can never fit
            q.state = GP_REQ_FAILED;
            q.error = GP_ERR_OOM;
            b->queue.pop_front();
            continue;
        }
        if (b->used_bytes + q.bytes > b->max_bytes) break;
        // enough work in flight to fill the GPU: later requests wait, so earlier
        // ones get more of the GPU and finish sooner (arrival order is kept)
        if (b->max_sites > 0 && running_count(b) > 0 &&
            running_sites(b) + (long long)q.p.nx * q.p.ny > b->max_sites)
            break;
        gp_handle* h = nullptr;
        int st = gp_create(&q.p, b->stream, &h);
        // The device is fuller than the accounting: wait for retirements while
        // solves are running; with none running nothing will free memory, so the
        // request fails (out of memory) instead of waiting forever.
        if (st == GP_ERR_OOM && running_count(b) > 0) break;
        b->queue.pop_front();
        if (st != GP_OK) {
            q.state = GP_REQ_FAILED;
            q.error = st;
            continue;
        }
        if ((st = gp_init_gaussian(h, q.r.frac, q.r.seed, q.r.phase_noise)) != GP_OK ||
            (st = ensure_coef(h, GP_IMAG)) != GP_OK) {
            gp_destroy(h);
            q.state = GP_REQ_FAILED;
            q.error = st;
            continue;
        }
        q.h = h;
        q.state = GP_REQ_RUNNING;
        b->used_bytes += q.bytes;
    }
    return GP_OK;
}

}  // namespace

extern "C" {

size_t gp_request_bytes(const gp_params* params, int policy)
{
    if (!params || validate(params) != GP_OK) return 0;
    gp_params p = *params;
    p.precision = policy_precision(policy);
    return handle_bytes(p);
}

int gp_batch_create(size_t max_device_bytes, int check_every, void* cuda_stream, gp_batch** out)
{
    if (!out || max_device_bytes == 0 || check_every <= 0) return GP_ERR_ARG;
    *out = nullptr;
    gp_batch* b = new (std::nothrow) gp_batch();
    if (!b) return GP_ERR_OOM;
    b->max_bytes = max_device_bytes;
    b->check_every = check_every;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return GP_ERR_CUDA;
        }
        b->own_stream = true;
    }
    if (!dalloc(&b->counts, 2 * kGroupCounts * sizeof(int)) || !dalloc(&b->flag, sizeof(int)) ||
        !dalloc(&b->work, 4 * sizeof(int)) || cudaMemsetAsync(b->flag, 0, sizeof(int), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->work, 0, 4 * sizeof(int), b->stream) != cudaSuccess) {
        gp_batch_destroy(b);
        return GP_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&b->stream32, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        gp_batch_destroy(b);
        return GP_ERR_CUDA;
    }
    *out = b;
    return GP_OK;
}

void gp_batch_destroy(gp_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& kv : b->reqs)
        if (kv.second.h) gp_destroy(kv.second.h);
    if (b->stream32) cudaStreamSynchronize(b->stream32);
    b->g64.release();
    b->g32.release();
    cudaFree(b->counts);
    cudaFree(b->work);
    cudaFree(b->flag);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->stream32) cudaStreamDestroy(b->stream32);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

int gp_batch_submit(gp_batch* b, const gp_params* params, const gp_request* req, long long* id_out)
{
    if (!b || !params || !req || !id_out) return GP_ERR_ARG;
    int st = validate(params);
    if (st) return st;
    if (req->policy != GP_POLICY_FP64 && req->policy != GP_POLICY_FP32_REFINE) return GP_ERR_ARG;
    if (!(req->tol > 0) || req->cap <= 0 || req->refine_steps < 0 || !std::isfinite(req->phase_noise))
        return GP_ERR_ARG;
    if (b->max_queued > 0 && (int)b->queue.size() >= b->max_queued) return GP_ERR_QUEUE_FULL;
    Request q;
    q.id = b->next_id++;
    q.p = *params;
    q.p.precision = policy_precision(req->policy);
    q.r = *req;
    q.bytes = handle_bytes(q.p);
    b->reqs[q.id] = q;
    b->queue.push_back(q.id);
    *id_out = q.id;
    return GP_OK;
}

int gp_batch_step(gp_batch* b, int* n_running, int* n_queued)
{
    gpspin::TraceRange trace("gp_batch_step");
    if (!b) return GP_ERR_ARG;
    int st = admit(b);
    if (st) return st;
    b->g64.clear();
    b->g32.clear();
    std::vector<Request*> run;
    for (auto& kv : b->reqs)
        if (kv.second.state == GP_REQ_RUNNING) run.push_back(&kv.second);
    // largest grids first: their work items (the longest lines) head the lists,
    // which a persistent launch hands out in order (longest jobs first)
    std::vector<Request*> order(run);
    std::stable_sort(order.begin(), order.end(), [](const Request* a, const Request* c) {
        return (long long)a->p.nx * a->p.ny > (long long)c->p.nx * c->p.ny;
    });
    for (Request* qp : order) {
        Request& q = *qp;
        const CoefSet& cs = q.h->coef[GP_IMAG];
        // batched launches use the unsplit tilings (no clusters in the work list)
        if (q.h->active == GP_FP32_MIXED) {
            PassArgsF ax = pass_args_f32(q.h, cs, 0), ay = pass_args_f32(q.h, cs, 1);
            ax.t = with_bulk(cs.fux, ax.t.bulk);
            ay.t = with_bulk(cs.fuy, ay.t.bulk);
            add_instance(b->g32, q.h, ax, ay);
        } else {
            PassArgs ax = pass_args(q.h, cs, 0), ay = pass_args(q.h, cs, 1);
            ax.t = with_bulk(cs.ux, ax.t.bulk);
            ay.t = with_bulk(cs.uy, ay.t.bulk);
            add_instance(b->g64, q.h, ax, ay);
        }
    }
    const int k = b->check_every;
    if (!run.empty()) {
        // the complex64 group runs on its own stream, after everything the
        // handles enqueued on the batch stream, and the batch stream waits for it
        BK(cudaEventRecord(b->ev_fork, b->stream));
        BK(cudaStreamWaitEvent(b->stream32, b->ev_fork, 0));
        if ((st = upload_and_run(b, b->g64, b->counts, b->work, k, b->stream))) return st;
        if ((st = upload_and_run(b, b->g32, b->counts + kGroupCounts, b->work + 2, k, b->stream32))) return st;
        BK(cudaEventRecord(b->ev_join, b->stream32));
        BK(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
        BK(cudaStreamSynchronize(b->stream));
    }
    // convergence checks between ticks
    for (Request* q : run) {
        q->h->scale_pending = true;
        q->h->steps += k;
        q->steps += k;
        gp_obs o;
        int ost = gp_observables(q->h, &o);
        q->obs = o;
        if (ost != GP_OK) {
            q->error = ost;
            retire(b, *q, GP_REQ_FAILED);
            continue;
        }
        const double de = q->have_e ? std::fabs(o.energy - q->e_last) : INFINITY;
        q->have_e = true;
        q->e_last = o.energy;
        if (q->h->active == GP_FP32_MIXED) {
            // FP32 phase: hand over to FP64 once the energy has settled to the FP32
            // level, and in any case early enough for a final FP64 refinement block
            if (de <= q->r.tol32 * std::fabs(o.energy) || q->steps + q->r.refine_steps >= q->r.cap) {
                if ((ost = gp_refine_fp64(q->h, 0, GP_IMAG)) != GP_OK) {
                    q->error = ost;
                    retire(b, *q, GP_REQ_FAILED);
                    continue;
                }
                q->have_e = false;  // restart the |dE| test in FP64
            }
            if (q->steps < q->r.cap) continue;
        }
        if (de < q->r.tol || q->steps >= q->r.cap) retire(b, *q, GP_REQ_DONE);
    }
    st = admit(b);  // memory freed by retirements
    if (n_running || n_queued) {
        int nr = 0;
        for (auto& kv : b->reqs) nr += kv.second.state == GP_REQ_RUNNING;
        if (n_running) *n_running = nr;
        if (n_queued) *n_queued = (int)b->queue.size();
    }
    return st;
}

int gp_batch_use_graphs(gp_batch* b, int enable)
{
    if (!b) return GP_ERR_ARG;
    b->graphs = enable != 0;
    if (!b->graphs) {
        b->g64.drop_graph();
        b->g32.drop_graph();
    }
    return GP_OK;
}

int gp_batch_set_persistent(gp_batch* b, int max_ctas)
{
    if (!b) return GP_ERR_ARG;
    const int v = max_ctas < 0 ? -1 : max_ctas;
    if (b->persist != v) {
        b->g64.drop_graph();  // the captured ticks hold the other launch form
        b->g32.drop_graph();
    }
    b->persist = v;
    return GP_OK;
}

int gp_batch_set_running_limit(gp_batch* b, long long max_sites)
{
    if (!b || max_sites < 0) return GP_ERR_ARG;
    b->max_sites = max_sites;
    return GP_OK;
}

int gp_batch_set_queue_limit(gp_batch* b, int max_queued)
{
    if (!b || max_queued < 0) return GP_ERR_ARG;
    b->max_queued = max_queued;
    return GP_OK;
}

int gp_batch_cancel(gp_batch* b, long long id)
{
    if (!b) return GP_ERR_ARG;
    auto it = b->reqs.find(id);
    if (it == b->reqs.end()) return GP_ERR_ARG;
    Request& q = it->second;
    if (q.state == GP_REQ_QUEUED) {
        b->queue.erase(std::remove(b->queue.begin(), b->queue.end(), id), b->queue.end());
        q.state = GP_REQ_CANCELLED;
    } else if (q.state == GP_REQ_RUNNING) {
        // between ticks no work of the solve is in flight: its memory is freed now
        // and the next gp_batch_step can admit into it
        if (q.h) {
            gp_destroy(q.h);
            q.h = nullptr;
            b->used_bytes -= q.bytes;
        }
        q.state = GP_REQ_CANCELLED;
    }
    return GP_OK;
}

int gp_batch_error(gp_batch* b, long long id)
{
    if (!b) return GP_ERR_ARG;
    auto it = b->reqs.find(id);
    return it == b->reqs.end() ? GP_ERR_ARG : it->second.error;
}

int gp_batch_poll(gp_batch* b, long long id, int* state, long long* steps, gp_obs* obs, double* psi_out, int release)
{
    if (!b) return GP_ERR_ARG;
    auto it = b->reqs.find(id);
    if (it == b->reqs.end()) {
        if (state) *state = GP_REQ_UNKNOWN;
        return GP_ERR_ARG;
    }
    Request& q = it->second;
    if (state) *state = q.state;
    if (steps) *steps = q.steps;
    if (obs) *obs = q.obs;
    if (q.state == GP_REQ_DONE && psi_out && !q.psi.empty())
        std::copy(q.psi.begin(), q.psi.end(), psi_out);
    if (release && (q.state == GP_REQ_DONE || q.state == GP_REQ_FAILED || q.state == GP_REQ_CANCELLED))
        b->reqs.erase(it);
    return GP_OK;
}

}  // extern "C"
