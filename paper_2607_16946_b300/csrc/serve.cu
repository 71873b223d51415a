// sdf_serve_*: a request loop over several resident clouds (the serving use
// of Sec. 6's applications: batches of SDF queries of uneven size, sphere-
// tracing steps, offsets and Booleans, against clouds kept on the device).
//
// Continuous batching: a scheduler thread admits queued requests (in arrival
// order, or smallest first with an age guard) whenever a slot (max_inflight)
// and enough of the memory budget are free, and launches each admitted request at once on one of n_streams CUDA
// streams, so requests that arrive while others run overlap with them on the
// device.  Completion is signalled by a host callback enqueued behind the
// request's work (no polling of the GPU); the scheduler then returns the
// request's memory to the budget and admits the next ones.
//
// A request's work depends only on its own inputs, cloud and options (the
// launch plan is a function of Q, N and the SM count), so its result is the
// same whether it runs alone or in a mix.
//
// Large requests are cut into query chunks (split_gpairs of the config): a
// ticket names a job, and a job of more (query, point) pairs than the budget
// runs as chunks of at least one full wave of unsplit query blocks on either
// engine (2 x resident blocks x SMs x 512 queries), so that every query's
// arithmetic is exactly that of the unsplit call.  A chunk's successor is
// queued at the tail when the chunk is admitted: other requests interleave
// with the chunks of a large one instead of waiting for all of it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace ptsdf {

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

__global__ void k_serve_positions(const float* __restrict__ org, const float* __restrict__ dir,
                                  const float* __restrict__ t, int64_t q, float* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    const float ti = t[i];
    for (int k = 0; k < 3; ++k) x[3 * i + k] = fmaf(ti, dir[3 * i + k], org[3 * i + k]);
}

__global__ void k_serve_combine(int op, const float* __restrict__ a, const float* __restrict__ b, int64_t q,
                                float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    const float x = a[i], y = b[i];
    out[i] = op == SDF_REQ_UNION ? fminf(x, y) : op == SDF_REQ_INTERSECT ? fmaxf(x, y) : fmaxf(x, -y);
}

// A submitted request (what a ticket names), run as `chunks` query chunks.
struct Job {
    uint64_t ticket = 0;
    sdf_request r{};
    sdf_request_stats st{};         // of the whole job; st.chunks = chunks
    int chunks = 1;
    int issued = 0;                 // chunks queued so far
    int remaining = 1;              // chunks not finished
    int64_t chunk_q = 0;            // queries per chunk (the last one takes the rest)
    bool finished = false;          // stats final, waiting for poll
};

// One schedulable unit: a job, or one chunk of it (queries [q0, q0 + q)).
struct Request {
    std::shared_ptr<Job> job;
    int64_t q0 = 0, q = 0;
    int64_t need = 0;               // bytes charged against the budget
    double work = 0.0;              // (query, point) pairs, for smallest-first admission
    int32_t status = SDF_OK;
    int64_t queued_ns = 0;          // when it joined the queue (the age guard of SMALLEST_FIRST)
    int64_t done_ns = 0;
    int stream = 0;
    bool bulk = false;              // above express_gpairs (when the server has express streams)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::atomic<bool> done{false};
};

struct Server {
    sdf_serve_config cfg{};
    std::vector<cudaStream_t> streams;
    std::vector<const Cloud*> clouds;
    std::mutex mu;
    std::condition_variable cv;     // scheduler wake-up
    std::condition_variable done_cv;  // pollers
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> inflight;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> all;
    int64_t mem_in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<double> stream_work;   // pairs of the requests in flight on each stream
    int n_express = 0;                 // streams [0, n_express) take the express class
    int bulk_inflight = 0;             // bulk requests in flight (at most max_inflight - max_inflight / 2)
    std::thread worker;
};

// bytes a request (or a chunk of q of its queries) needs on the device:
// staging of host buffers plus the scratch of the query kernels for its plan
int64_t request_need(const Server& S, const sdf_request& r, int64_t q) {
    int64_t b = 0;
    auto scratch = [&](const Cloud* c, bool grad) -> int64_t {
        if (r.opts.lambda_mode == SDF_LAMBDA_RADIUS) return q * 8 + 4096;   // the fallback list
        const Plan p = make_plan(*c, q, r.opts.split_n, grad ? kConsumerWarps * 32 : kQueriesPerCta);
        int64_t s = (int64_t)p.split * q * 8;                 // prepass partials
        if (grad) {
            s += (int64_t)p.split * q * 4 + (p.split > 1 ? (int64_t)p.split * q * 52 : 0);
        } else {
            const int parts = query_partials(*c, q, r.opts);   // (W, S) partial rows
            if (parts > 1) s += (int64_t)parts * q * 8;
        }
        return s + 4096;
    };
    const Cloud* ca = S.clouds[r.cloud_id];
    switch (r.kind) {
        case SDF_REQ_QUERY:
            b = scratch(ca, false) + (r.host_buffers ? q * 16 : 0);
            break;
        case SDF_REQ_GRAD:
            b = scratch(ca, true) + q * 12 + (r.host_buffers ? q * 28 : 0);
            break;
        case SDF_REQ_TRACE_STEP:
            b = scratch(ca, false) + q * 12 + (r.host_buffers ? q * 32 : 0);
            break;
        default: {   // Booleans: two queries and two phi buffers
            const Cloud* cb = S.clouds[r.cloud_id_b];
            b = std::max(scratch(ca, false), scratch(cb, false)) + q * 8 + (r.host_buffers ? q * 16 : 0);
        }
    }
    return b;
}

void CUDART_CB on_request_done(void* p) {
    // Runs on a CUDA driver thread once the request's work is complete.  It
    // takes no lock and makes no CUDA call; a wake-up that races the
    // scheduler's wait is covered by the scheduler's short wait timeout.
    auto* pr = static_cast<std::pair<Server*, Request*>*>(p);
    Server* S = pr->first;
    Request* R = pr->second;
    delete pr;
    R->done_ns = now_ns();
    R->done.store(true, std::memory_order_release);
    S->cv.notify_all();
}

unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

// The stream of a request of `work` pairs: within its priority class (the
// express streams for small requests when express_gpairs > 0), the one with
// the least work in flight, so a request never waits in a stream's order
// behind a larger one while another stream of its class has less.
bool is_bulk(const Server& S, double work) {
    return S.n_express > 0 && work > (double)S.cfg.express_gpairs * 1e9;
}

int pick_stream(const Server& S, double work) {
    int lo = 0, hi = (int)S.streams.size();
    if (S.n_express > 0) {
        if (is_bulk(S, work))
            lo = S.n_express;
        else
            hi = S.n_express;
    }
    int best = lo;
    for (int i = lo + 1; i < hi; ++i)
        if (S.stream_work[i] < S.stream_work[best]) best = i;
    return best;
}

// Enqueues one admitted request (or chunk) on its stream.
sdf_status launch_request(Server& S, Request& R) {
    cudaStream_t st = S.streams[R.stream];
    // the chunk's view of the job's buffers (a GRAD job is never cut)
    sdf_request r = R.job->r;
    const int64_t q = R.q;
    if (R.q0 > 0) {
        r.x += 3 * R.q0;
        r.out += R.q0;
        if (r.dirs) r.dirs += 3 * R.q0;
        if (r.t) r.t += R.q0;
    }
    r.q = q;
    const Cloud& ca = *S.clouds[r.cloud_id];
    cudaError_t e = cudaEventRecord(R.ev0, st);
    if (e != cudaSuccess) return cuda_error(e, "serve: event");
    std::vector<void*> tmp;
    auto dalloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocAsync(p, bytes, st);
        if (e == cudaSuccess) tmp.push_back(*p);
    };
    sdf_status s = SDF_OK;
    const float* x = r.x;
    float* out = r.out;
    float* dx = nullptr;
    float* dout = nullptr;
    const int64_t out_floats = r.kind == SDF_REQ_GRAD ? 4 * q : q;
    if (r.host_buffers) {
        const int64_t in_floats = r.kind == SDF_REQ_TRACE_STEP ? 7 * q : 3 * q;
        dalloc((void**)&dx, (size_t)in_floats * 4);
        dalloc((void**)&dout, (size_t)out_floats * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dx, r.x, (size_t)q * 12, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && r.kind == SDF_REQ_TRACE_STEP) {
            e = cudaMemcpyAsync(dx + 3 * q, r.dirs, (size_t)q * 12, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dx + 6 * q, r.t, (size_t)q * 4, cudaMemcpyHostToDevice, st);
        }
        x = dx;
        out = dout;
    }
    if (e != cudaSuccess) s = cuda_error(e, "serve: staging");
    if (s == SDF_OK) {
        switch (r.kind) {
            case SDF_REQ_QUERY:
                s = launch_query(ca, x, q, out, r.opts, st);
                break;
            case SDF_REQ_GRAD:
                s = launch_query_grad(ca, x, q, out, out + q, nullptr, r.opts, st);
                break;
            case SDF_REQ_TRACE_STEP: {
                const float* org = x;
                const float* dir = r.host_buffers ? x + 3 * q : r.dirs;
                const float* tt = r.host_buffers ? x + 6 * q : r.t;
                float* pos = nullptr;
                dalloc((void**)&pos, (size_t)q * 12);
                if (e != cudaSuccess) {
                    s = cuda_error(e, "serve: scratch");
                    break;
                }
                k_serve_positions<<<nblk(q), 256, 0, st>>>(org, dir, tt, q, pos);
                s = launch_query(ca, pos, q, out, r.opts, st);
                break;
            }
            default: {
                const Cloud& cb = *S.clouds[r.cloud_id_b];
                float* pa = nullptr;
                float* pb = nullptr;
                dalloc((void**)&pa, (size_t)q * 4);
                dalloc((void**)&pb, (size_t)q * 4);
                if (e != cudaSuccess) {
                    s = cuda_error(e, "serve: scratch");
                    break;
                }
                s = launch_query(ca, x, q, pa, r.opts, st);
                if (s == SDF_OK) s = launch_query(cb, x, q, pb, r.opts, st);
                if (s == SDF_OK) k_serve_combine<<<nblk(q), 256, 0, st>>>(r.kind, pa, pb, q, out);
            }
        }
    }
    if (s == SDF_OK && r.host_buffers) {
        e = cudaMemcpyAsync(r.out, dout, (size_t)out_floats * 4, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) s = cuda_error(e, "serve: copy out");
    }
    for (void* p : tmp) cudaFreeAsync(p, st);
    cudaEventRecord(R.ev1, st);
    auto* arg = new std::pair<Server*, Request*>(&S, &R);
    e = cudaLaunchHostFunc(st, on_request_done, arg);
    if (e != cudaSuccess) {
        // no callback will come: wait for the stream here and finish the request
        delete arg;
        cudaStreamSynchronize(st);
        R.done_ns = now_ns();
        R.done.store(true, std::memory_order_release);
        return cuda_error(e, "serve: completion callback");
    }
    return s;
}

// Queries of one launch plan with no point split on either engine: two waves
// of the FP32-unit loop's query blocks (the tensor-core loop needs fewer).
int64_t min_chunk_queries(const Cloud& c) { return 2LL * kFwdMinBlocks * c.num_sms * kQueriesPerCta; }

// The job's next chunk as a schedulable request (queries and charges).
std::shared_ptr<Request> make_chunk(const Server& S, const std::shared_ptr<Job>& job) {
    Job& J = *job;
    auto R = std::make_shared<Request>();
    R->job = job;
    R->q0 = (int64_t)J.issued * J.chunk_q;
    R->q = J.issued + 1 < J.chunks ? J.chunk_q : J.r.q - R->q0;
    const sdf_request& r = J.r;
    const bool two = r.kind == SDF_REQ_UNION || r.kind == SDF_REQ_INTERSECT || r.kind == SDF_REQ_DIFFERENCE;
    R->need = request_need(S, r, R->q);
    R->work = (double)R->q * (double)(S.clouds[r.cloud_id]->n + (two ? S.clouds[r.cloud_id_b]->n : 0));
    R->queued_ns = J.issued == 0 ? J.st.arrive_ns : now_ns();
    ++J.issued;
    return R;
}

void scheduler(Server* S) {
    cudaSetDevice(S->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // retire finished requests and chunks; a job is finished with its last chunk
        for (auto it = S->inflight.begin(); it != S->inflight.end();) {
            Request& R = **it;
            if (R.done.load(std::memory_order_acquire)) {
                Job& J = *R.job;
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, R.ev0, R.ev1) == cudaSuccess) J.st.device_ms += ms;
                cudaEventDestroy(R.ev0);
                cudaEventDestroy(R.ev1);
                S->mem_in_use -= R.need;
                S->stream_work[R.stream] -= R.work;
                if (R.bulk) --S->bulk_inflight;
                if (R.status != SDF_OK && J.st.status == SDF_OK) J.st.status = R.status;
                J.st.done_ns = std::max(J.st.done_ns, R.done_ns);
                if (--J.remaining == 0) {
                    J.finished = true;
                    S->done_cv.notify_all();
                }
                it = S->inflight.erase(it);
            } else {
                ++it;
            }
        }
        // admit while a slot and the memory are free: the head of the queue
        // (FIFO, or a request older than starve_ms), else the smallest request.
        // With express streams, bulk requests hold at most the slots that
        // max_inflight / 2 leaves, so a small request never waits for a slot
        // behind large ones that share the device at low priority.
        while (!S->queue.empty() && (int)S->inflight.size() < S->cfg.max_inflight) {
            const bool bulk_full = S->n_express > 0 &&
                                   S->bulk_inflight >= S->cfg.max_inflight - S->cfg.max_inflight / 2;
            auto admissible = [&](const Request& R) { return !(bulk_full && is_bulk(*S, R.work)); };
            size_t pick = S->queue.size();
            const bool starving = now_ns() - S->queue.front()->queued_ns > (int64_t)S->cfg.starve_ms * 1000000LL;
            for (size_t i = 0; i < S->queue.size(); ++i) {
                if (!admissible(*S->queue[i])) continue;
                if (pick == S->queue.size()) {
                    pick = i;
                    if (S->cfg.policy != SDF_SERVE_SMALLEST_FIRST || (i == 0 && starving)) break;
                } else if (S->queue[i]->work < S->queue[pick]->work) {
                    pick = i;
                }
            }
            if (pick == S->queue.size()) break;
            if (S->mem_in_use + S->queue[pick]->need > S->cfg.mem_budget_bytes) break;
            std::shared_ptr<Request> R = S->queue[pick];
            S->queue.erase(S->queue.begin() + (long)pick);
            Job& J = *R->job;
            if (R->q0 == 0) J.st.admit_ns = now_ns();
            R->stream = pick_stream(*S, R->work);
            R->bulk = is_bulk(*S, R->work);
            if (R->bulk) ++S->bulk_inflight;
            S->stream_work[R->stream] += R->work;
            S->mem_in_use += R->need;
            cudaEventCreate(&R->ev0);
            cudaEventCreate(&R->ev1);
            if (R->q0 == 0) J.st.start_ns = now_ns();
            R->status = launch_request(*S, *R);
            S->inflight.push_back(R);
            if (J.issued < J.chunks) S->queue.push_back(make_chunk(*S, R->job));   // the next chunk, at the tail
        }
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;
        S->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

}  // namespace

}  // namespace ptsdf

using namespace ptsdf;

struct sdf_server_s {
    Server s;
};

extern "C" sdf_status sdf_serve_create(const sdf_serve_config* cfg, sdf_server* out) {
    if (!cfg || !out) return set_error(SDF_EINVAL, "sdf_serve_create: NULL argument");
    *out = nullptr;
    if (cfg->max_inflight < 1 || cfg->n_streams < 1 || cfg->mem_budget_bytes < 1)
        return set_error(SDF_EINVAL, "sdf_serve_create: need max_inflight >= 1, n_streams >= 1, budget > 0");
    if ((cfg->policy != SDF_SERVE_FIFO && cfg->policy != SDF_SERVE_SMALLEST_FIRST) || cfg->starve_ms < 0)
        return set_error(SDF_EINVAL, "sdf_serve_create: unknown policy or negative starve_ms");
    if (!(cfg->express_gpairs >= 0.f) || (cfg->express_gpairs > 0.f && cfg->n_streams < 2))
        return set_error(SDF_EINVAL, "sdf_serve_create: express_gpairs must be >= 0, and > 0 needs n_streams >= 2");
    auto* h = new sdf_server_s();
    Server& S = h->s;
    S.cfg = *cfg;
    cudaError_t e = cudaSetDevice(cfg->device);
    // express streams at the highest priority, the others at the lowest
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    S.n_express = cfg->express_gpairs > 0.f ? cfg->n_streams / 2 : 0;
    for (int i = 0; e == cudaSuccess && i < cfg->n_streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, i < S.n_express ? greatest : least);
        if (e == cudaSuccess) S.streams.push_back(st);
    }
    S.stream_work.assign(S.streams.size(), 0.0);
    if (e != cudaSuccess) {
        for (auto st : S.streams) cudaStreamDestroy(st);
        delete h;
        return cuda_error(e, "sdf_serve_create");
    }
    S.worker = std::thread(scheduler, &S);
    *out = h;
    return SDF_OK;
}

extern "C" sdf_status sdf_serve_register(sdf_server srv, sdf_cloud cloud, int32_t* cloud_id) {
    if (!srv || !cloud || !cloud_id) return set_error(SDF_EINVAL, "sdf_serve_register: NULL argument");
    Server& S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    *cloud_id = (int32_t)S.clouds.size();
    S.clouds.push_back(reinterpret_cast<const Cloud*>(cloud));
    return SDF_OK;
}

extern "C" sdf_status sdf_serve_submit(sdf_server srv, const sdf_request* req, uint64_t* ticket) {
    if (!srv || !req || !ticket) return set_error(SDF_EINVAL, "sdf_serve_submit: NULL argument");
    Server& S = srv->s;
    const int64_t t_arrive = now_ns();
    const sdf_request& r = *req;
    if (r.q < 1) return set_error(SDF_EINVAL, "sdf_serve_submit: q must be >= 1");
    if (r.kind < SDF_REQ_QUERY || r.kind > SDF_REQ_TRACE_STEP)
        return set_error(SDF_EINVAL, "sdf_serve_submit: unknown request kind");
    if (!r.x || !r.out || (r.kind == SDF_REQ_TRACE_STEP && (!r.dirs || !r.t)))
        return set_error(SDF_EINVAL, "sdf_serve_submit: NULL buffer");
    if ((r.opts.precision != SDF_F32 && r.opts.precision != SDF_F16X2 && r.opts.precision != SDF_BF16X2) ||
        (r.kind == SDF_REQ_GRAD && r.opts.precision != SDF_F32) || !(r.opts.C > 0.f) || r.opts.split_n < 0 ||
        (r.opts.engine != SDF_ENGINE_AUTO && r.opts.engine != SDF_ENGINE_ALU && r.opts.engine != SDF_ENGINE_TENSOR) ||
        (r.opts.engine == SDF_ENGINE_TENSOR && (r.opts.precision != SDF_F32 || r.kind == SDF_REQ_GRAD)) ||
        (r.opts.lambda_mode != SDF_LAMBDA_GLOBAL && r.opts.lambda_mode != SDF_LAMBDA_FIXED &&
         r.opts.lambda_mode != SDF_LAMBDA_RADIUS) ||
        (r.opts.lambda_mode == SDF_LAMBDA_RADIUS &&
         (r.kind == SDF_REQ_GRAD || !(r.opts.fixed_lambda > 0.f) || r.opts.precision != SDF_F32 ||
          r.opts.engine == SDF_ENGINE_TENSOR)) ||
        (r.opts.formula != SDF_FORMULA_BLEND && r.opts.formula != SDF_FORMULA_LSE) ||
        (r.opts.formula == SDF_FORMULA_LSE &&
         (r.kind != SDF_REQ_QUERY || (r.opts.lambda_mode == SDF_LAMBDA_FIXED && !(r.opts.fixed_lambda > 0.f)))))
        return set_error(SDF_EINVAL, "sdf_serve_submit: bad options");
    auto J = std::make_shared<Job>();
    J->r = r;
    J->st.arrive_ns = t_arrive;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        const bool two = r.kind == SDF_REQ_UNION || r.kind == SDF_REQ_INTERSECT || r.kind == SDF_REQ_DIFFERENCE;
        if (r.cloud_id < 0 || r.cloud_id >= (int32_t)S.clouds.size() ||
            (two && (r.cloud_id_b < 0 || r.cloud_id_b >= (int32_t)S.clouds.size())))
            return set_error(SDF_EINVAL, "sdf_serve_submit: unknown cloud id");
        if (S.stop) return set_error(SDF_EBUSY, "sdf_serve_submit: server is shutting down");
        // cut a large job into chunks of at least min_chunk_queries each
        const Cloud& ca = *S.clouds[r.cloud_id];
        const double pairs = (double)r.q * (double)(ca.n + (two ? S.clouds[r.cloud_id_b]->n : 0));
        if (S.cfg.split_gpairs > 0 && r.kind != SDF_REQ_GRAD && pairs > S.cfg.split_gpairs * 1e9) {
            const int64_t most = r.q / (min_chunk_queries(ca) + kQueriesPerCta);
            const double want = std::ceil(pairs / (S.cfg.split_gpairs * 1e9));
            J->chunks = (int)std::max<int64_t>(1, std::min<int64_t>(most, (int64_t)std::min(want, 1e6)));
        }
        J->chunk_q = J->chunks > 1 ? (r.q / J->chunks) / kQueriesPerCta * kQueriesPerCta : r.q;
        J->remaining = J->chunks;
        J->st.chunks = J->chunks;
        // the largest chunk (the last) must fit the budget on its own
        const int64_t last_q = r.q - (int64_t)(J->chunks - 1) * J->chunk_q;
        const int64_t need = request_need(S, r, last_q);
        if (need > S.cfg.mem_budget_bytes)
            return set_error(SDF_ENOMEM, "sdf_serve_submit: request needs " + std::to_string(need) +
                                             " bytes, more than the whole memory budget");
        J->ticket = S.next_ticket++;
        S.all[J->ticket] = J;
        S.queue.push_back(make_chunk(S, J));
        *ticket = J->ticket;
    }
    S.cv.notify_all();
    return SDF_OK;
}

extern "C" sdf_status sdf_serve_poll(sdf_server srv, uint64_t ticket, int64_t timeout_us,
                                     sdf_request_stats* stats) {
    if (!srv) return set_error(SDF_EINVAL, "sdf_serve_poll: NULL server");
    Server& S = srv->s;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.all.find(ticket);
    if (it == S.all.end()) return set_error(SDF_EINVAL, "sdf_serve_poll: unknown ticket");
    std::shared_ptr<Job> J = it->second;
    if (timeout_us < 0) {
        S.done_cv.wait(lk, [&] { return J->finished; });
    } else {
        // clamp to a day so that the deadline cannot overflow the clock
        const int64_t us = std::min<int64_t>(timeout_us, 86400LL * 1000000LL);
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(us);
        while (!J->finished) {
            if (S.done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !J->finished)
                return set_error(SDF_ETIMEOUT, "sdf_serve_poll: not finished");
        }
    }
    if (stats) *stats = J->st;
    S.all.erase(it);
    return J->st.status == SDF_OK ? SDF_OK : (sdf_status)J->st.status;
}

extern "C" sdf_status sdf_serve_stats(sdf_server srv, int32_t* queued, int32_t* inflight, int64_t* mem_in_use) {
    if (!srv) return set_error(SDF_EINVAL, "sdf_serve_stats: NULL server");
    Server& S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    if (queued) *queued = (int32_t)S.queue.size();
    if (inflight) *inflight = (int32_t)S.inflight.size();
    if (mem_in_use) *mem_in_use = S.mem_in_use;
    return SDF_OK;
}

extern "C" sdf_status sdf_serve_shutdown(sdf_server srv) {
    if (!srv) return SDF_OK;
    Server& S = srv->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
    }
    S.cv.notify_all();
    if (S.worker.joinable()) S.worker.join();
    for (auto st : S.streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete srv;
    return SDF_OK;
}
