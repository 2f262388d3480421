// serve.cu -- tc_submit / tc_poll: a continuous-batching request server.
//
// Requests go to one of two lanes by size.  The small lane has two worker
// threads, the large lane one; every worker has a private sub-context (own
// stream, arenas and control block).  A worker takes queued requests of its
// lane into its next round while (a) their estimated scratch fits the device
// memory free at that moment (cudaMemGetInfo, read before every round, split
// across the workers) plus what the worker's arenas already hold, and (b) the
// round stays below a work bound (undirected edges), so that no round -- and
// no request queued behind one -- waits for an unbounded batch.  It counts the
// round with the batched union pipeline (one graph: tc_count directly),
// publishes every request of the round with its latency, and immediately
// admits whatever arrived meanwhile.  While one worker's round runs on the
// device the others admit and launch theirs, so rounds overlap on the GPU,
// and a large graph (the large lane) never holds up the small requests
// behind it.
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
    std::condition_variable cv[2];
    std::deque<uint64_t> queue[2];  // lane 0: small requests, lane 1: large ones
    std::unordered_map<uint64_t, ServeRequest> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    uint32_t max_batch = 4096;           // graphs per round
    uint64_t round_edges = 1ull << 25;   // small lane: undirected edges per round (the first request always fits)
    uint64_t large_slots = 1ull << 23;   // a graph with more CSR slots goes to the large lane
    double mem_fraction = 0.8;           // share of the free device memory the workers may grow into
    std::vector<tc_ctx *> subs;
    std::vector<int> lane;
    std::vector<std::thread> workers;
    size_t queued() const { return queue[0].size() + queue[1].size(); }
};

namespace tc {

static size_t request_bytes(const tc_ctx *sub, const tc_graph *g) {
    uint64_t hs = 0;
    uint32_t hb = 0;
    // union copy + per-vertex scratch; the hub tables are shared per round
    return pipeline_bytes(sub, g->n, g->slots, 0, true, true, &hs, &hb) + 8ull * (g->n + 1) + 4ull * (g->slots + 1);
}

static size_t arena_held(const tc_ctx *sub) { return sub->arena.cap + sub->batch_arena.cap; }

static void worker_loop(ServeState *S, tc_ctx *sub, int lane, int nworkers) {
    cudaSetDevice(sub->device);
    std::vector<uint64_t> tickets;
    std::vector<const tc_graph *> graphs;
    std::vector<uint64_t> out;
    for (;;) {
        tickets.clear();
        graphs.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv[lane].wait(lk, [&] { return S->stop || !S->queue[lane].empty(); });
            if (S->stop && S->queue[lane].empty()) return;
        }
        // memory for this round: what the worker's arenas hold plus its share of
        // what is free on the device right now
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            free_b = 0;
        }
        const size_t budget = arena_held(sub) + (size_t)(free_b * S->mem_fraction) / (size_t)nworkers;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            std::deque<uint64_t> &q = S->queue[lane];
            size_t used = 0;
            uint64_t edges = 0;
            while (!q.empty() && tickets.size() < S->max_batch) {
                const uint64_t t = q.front();
                ServeRequest &rq = S->reqs[t];
                const size_t b = request_bytes(sub, rq.g);
                const uint64_t e = rq.g->slots / 2;
                // a large-lane round is one graph; a small-lane round stops at round_edges
                if (!tickets.empty() && (lane == 1 || used + b > budget || edges + e > S->round_edges)) break;
                used += b;
                edges += e;
                q.pop_front();
                rq.state = 1;
                tickets.push_back(t);
                graphs.push_back(rq.g);
            }
        }
        if (tickets.empty()) continue;
        out.assign(tickets.size(), 0);
        tc_status st;
        if (graphs.size() == 1) st = tc_count(sub, graphs[0], &out[0], nullptr);
        else st = tc_count_batch(sub, (uint32_t)graphs.size(), graphs.data(), out.data());
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
    const int lanes[] = {0, 0, 1};  // two small-lane workers, one large-lane worker
    const int nworkers = 3;
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
        if (lanes[i] == 1) {
            // the large lane's kernels get the device's highest stream priority: its
            // blocks are scheduled first whenever the small rounds' kernels leave room,
            // so a large count is not spread thin between many small rounds
            int least = 0, greatest = 0;
            cudaStream_t hs = nullptr;
            int prev = -1;
            cudaGetDevice(&prev);
            cudaSetDevice(ctx->device);
            if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
                cudaStreamCreateWithPriority(&hs, cudaStreamNonBlocking, greatest) == cudaSuccess) {
                cudaStreamDestroy(sub->own_stream);
                sub->own_stream = hs;
                sub->stream = hs;
            } else {
                cudaGetLastError();
            }
            if (prev >= 0) cudaSetDevice(prev);
        }
        S->subs.push_back(sub);
        S->lane.push_back(lanes[i]);
    }
    for (size_t i = 0; i < S->subs.size(); ++i) S->workers.emplace_back(worker_loop, S, S->subs[i], S->lane[i], nworkers);
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
    S->cv[0].notify_all();
    S->cv[1].notify_all();
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
    int lane = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queued() >= ctx->opt.max_queue) return TC_ERR_BUSY;
        const uint64_t t = S->next_ticket++;
        ServeRequest rq;
        rq.g = g;
        rq.t_submit = std::chrono::steady_clock::now();
        S->reqs.emplace(t, rq);
        lane = g->slots > S->large_slots ? 1 : 0;
        S->queue[lane].push_back(t);
        *ticket = t;
    }
    S->cv[lane].notify_one();
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
