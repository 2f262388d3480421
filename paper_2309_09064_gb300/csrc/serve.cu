// serve.cu -- tc_submit / tc_poll: a continuous-batching request server.
//
// Two worker threads, each with a private sub-context (own stream, arenas and
// control block), take requests from one queue.  A worker admits queued
// requests into its next round while their estimated scratch fits its memory
// budget (a share of the device memory free when serving started), counts
// the round with the batched union pipeline, publishes the results, and
// immediately admits whatever arrived meanwhile.  While one worker's round
// runs on the device the other admits and launches the next, so rounds
// overlap on the GPU and a request never waits for a full batch to form.
#include <chrono>

#include "pipeline.cuh"

struct ServeRequest {
    const tc_graph *g = nullptr;
    uint64_t result = 0;
    tc_status st = TC_OK;
    int state = 0;  // 0 queued, 1 running, 2 done
    std::chrono::steady_clock::time_point t_submit, t_done;
};

struct ServeState {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, ServeRequest> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t budget = 0;          // scratch bytes per round and worker
    uint32_t max_batch = 4096;  // graphs per round
    std::vector<tc_ctx *> subs;
    std::vector<std::thread> workers;
};

namespace tc {

static size_t request_bytes(const tc_ctx *sub, const tc_graph *g) {
    uint64_t hs = 0;
    uint32_t hb = 0;
    // union copy + per-vertex scratch; the hub tables are shared per round
    return pipeline_bytes(sub, g->n, g->slots, 0, true, &hs, &hb) + 8ull * (g->n + 1) + 4ull * (g->slots + 1);
}

static void worker_loop(ServeState *S, tc_ctx *sub) {
    std::vector<uint64_t> tickets;
    std::vector<const tc_graph *> graphs;
    std::vector<uint64_t> out;
    for (;;) {
        tickets.clear();
        graphs.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop && S->queue.empty()) return;
            size_t used = 0;
            while (!S->queue.empty() && tickets.size() < S->max_batch) {
                const uint64_t t = S->queue.front();
                ServeRequest &rq = S->reqs[t];
                const size_t b = request_bytes(sub, rq.g);
                if (!tickets.empty() && used + b > S->budget) break;  // admit when memory frees up
                used += b;
                S->queue.pop_front();
                rq.state = 1;
                tickets.push_back(t);
                graphs.push_back(rq.g);
            }
        }
        out.assign(tickets.size(), 0);
        tc_status st = tc_count_batch(sub, (uint32_t)graphs.size(), graphs.data(), out.data());
        {
            const auto now = std::chrono::steady_clock::now();
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t i = 0; i < tickets.size(); ++i) {
                auto it = S->reqs.find(tickets[i]);
                if (it == S->reqs.end()) continue;
                it->second.result = out[i];
                it->second.st = st;
                it->second.state = 2;
                it->second.t_done = now;
            }
        }
    }
}

static tc_status serve_start(tc_ctx *ctx) {
    ServeState *S = new ServeState();
    size_t free_b = 0, total_b = 0;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    const cudaError_t mem_e = cudaMemGetInfo(&free_b, &total_b);
    if (prev >= 0) cudaSetDevice(prev);
    if (mem_e != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return set_error(ctx, TC_ERR_CUDA, "cudaMemGetInfo failed");
    }
    const int nworkers = 2;
    S->budget = (size_t)(free_b * 0.6) / nworkers;
    for (int i = 0; i < nworkers; ++i) {
        tc_options o = ctx->opt;
        o.stream = nullptr;
        tc_ctx *sub = nullptr;
        if (tc_create(&sub, ctx->device, &o) != TC_OK) {
            for (tc_ctx *c : S->subs) tc_destroy(c);
            delete S;
            return set_error(ctx, TC_ERR_CUDA, "serving sub-context creation failed");
        }
        sub->tune = ctx->tune;
        S->subs.push_back(sub);
    }
    for (tc_ctx *sub : S->subs) S->workers.emplace_back(worker_loop, S, sub);
    ctx->serve = S;
    return TC_OK;
}

void serve_shutdown(tc_ctx *ctx) {
    ServeState *S = ctx->serve;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto &t : S->workers) t.join();
    for (tc_ctx *c : S->subs) tc_destroy(c);
    delete S;
    ctx->serve = nullptr;
}

}  // namespace tc

using namespace tc;

static std::mutex g_serve_start_mu;

extern "C" {

tc_status tc_submit(tc_ctx *ctx, const tc_graph *g, uint64_t *ticket) {
    if (!ctx || !g || !ticket) return TC_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(g_serve_start_mu);
        if (!ctx->serve) {
            tc_status st = serve_start(ctx);
            if (st != TC_OK) return st;
        }
    }
    ServeState *S = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.size() >= ctx->opt.max_queue) return TC_ERR_BUSY;
        const uint64_t t = S->next_ticket++;
        ServeRequest rq;
        rq.g = g;
        rq.t_submit = std::chrono::steady_clock::now();
        S->reqs.emplace(t, rq);
        S->queue.push_back(t);
        *ticket = t;
    }
    S->cv.notify_one();
    return TC_OK;
}

tc_status tc_poll_ex(tc_ctx *ctx, uint64_t ticket, uint64_t *triangles, uint64_t *latency_ns) {
    if (!ctx || !triangles) return TC_ERR_INVALID;
    ServeState *S = ctx->serve;
    if (!S) return TC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return TC_ERR_INVALID;
    if (it->second.state != 2) return TC_NOT_READY;
    const tc_status st = it->second.st;
    *triangles = it->second.result;
    if (latency_ns)
        *latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(it->second.t_done -
                                                                                     it->second.t_submit)
                          .count();
    S->reqs.erase(it);
    return st;
}

tc_status tc_poll(tc_ctx *ctx, uint64_t ticket, uint64_t *triangles) { return tc_poll_ex(ctx, ticket, triangles, nullptr); }

}  // extern "C"
