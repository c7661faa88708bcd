// drt_serve.cu -- a11: the request loop of the anticipative-prediction service.
//
// Requests (link, time grid, frequency grid, caller H buffer, optional record buffers) arrive from
// any thread.  One serving thread admits them by HBM footprint into an arena that the context
// reserved within its budget, and forms batches from whatever is queued when a slot (a stream) is
// free: continuous batching, so requests that arrive while other batches are on the GPU start as
// soon as a slot and memory free up, and their kernels overlap with the running ones.  A batch is a
// batch plan (drt_batch.cu) placed in an arena block; a host function queued behind its kernels
// stamps the completion time of its requests and hands the block back.  Link state stays resident:
// a request references a loaded link, whose unloading is refused while requests on it are pending.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "drt_internal.h"

namespace drt {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Server;

struct Slot {
    Server *srv = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    bool busy = false, completed = false;
    BatchPlan *plan = nullptr;
    size_t off = 0, size = 0;
    std::vector<uint64_t> tickets;
    unsigned long long *overflow = nullptr;   // pinned: the batch's FP64 redo-overflow word, copied behind it
};

struct Request {
    ServeItem item;
    drt_result res{};
    bool done = false;
};

struct Server {
    int device = 0;
    char *arena = nullptr;
    size_t arena_bytes = 0, arena_used = 0, arena_peak = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> size, coalesced
    int max_batch = 256;
    std::vector<Slot> slots;
    std::map<int, int> variant_of_bins;     // synthesis tile variant, tuned once per bin count
    std::mutex m;
    std::condition_variable cv, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    drt_serve_stats stats{};
    std::thread th;
    std::string fatal;   // a CUDA failure of the serving thread; later submissions report it

    // first fit in the arena (256-byte granules)
    bool arena_take(size_t bytes, size_t *off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            size_t rest = it->second - bytes, roff = it->first + bytes;
            free_blocks.erase(it);
            if (rest) free_blocks[roff] = rest;
            arena_used += bytes;
            arena_peak = std::max(arena_peak, arena_used);
            return true;
        }
        return false;
    }
    void arena_give(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        arena_used -= bytes;
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

// runs on CUDA's callback thread once a batch's kernels are done: no CUDA calls here
static void CUDART_CB on_batch_done(void *arg) {
    Slot *sl = static_cast<Slot *>(arg);
    Server *S = sl->srv;
    const double t = now_s();
    // a wave that queued more FP64 redo steps than its list holds left those steps out of H
    const drt_status st = (sl->overflow && *sl->overflow) ? DRT_ENOMEM : DRT_OK;
    {
        std::lock_guard<std::mutex> lk(S->m);
        for (uint64_t tk : sl->tickets) {
            auto it = S->reqs.find(tk);
            if (it == S->reqs.end()) continue;
            if (st != DRT_OK) it->second.res.status = st;
            it->second.res.t_done = t;
            it->second.done = true;
            it->second.item.inflight->fetch_sub(1);
            S->stats.completed++;
        }
        sl->completed = true;
    }
    S->cv.notify_all();
    S->cv_done.notify_all();
}

static void fail_requests(Server *S, const std::vector<uint64_t> &tickets, drt_status st) {
    const double t = now_s();
    std::lock_guard<std::mutex> lk(S->m);
    for (uint64_t tk : tickets) {
        auto it = S->reqs.find(tk);
        if (it == S->reqs.end()) continue;
        it->second.res.status = st;
        it->second.res.t_done = t;
        it->second.done = true;
        it->second.item.inflight->fetch_sub(1);
        S->stats.completed++;
    }
}

static void serve_loop(Server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        // 1. wait for work, a completed batch or the stop request
        std::vector<uint64_t> batch;
        std::vector<ServeItem> items;
        Slot *slot = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->m);
            S->cv.wait_for(lk, std::chrono::milliseconds(50), [&] {
                bool any_free = false, any_busy = false;
                for (auto &sl : S->slots) {
                    if (sl.completed) return true;
                    any_free = any_free || !sl.busy;
                    any_busy = any_busy || sl.busy;
                }
                if (!S->queue.empty() && any_free) return true;
                return S->stop && !any_busy;
            });
            // 2. hand back the blocks of finished batches
            for (auto &sl : S->slots)
                if (sl.completed) {
                    S->arena_give(sl.off, sl.size);
                    batch_free(sl.plan);   // the plan does not own its block
                    sl.plan = nullptr;
                    sl.tickets.clear();
                    sl.busy = sl.completed = false;
                }
            bool any_busy = false;
            for (auto &sl : S->slots) any_busy = any_busy || sl.busy;
            if (S->stop && S->queue.empty() && !any_busy) return;
            for (auto &sl : S->slots)
                if (!sl.busy) {
                    slot = &sl;
                    break;
                }
            // 3. take the queued requests in arrival order, up to max_batch
            if (slot)
                while (!S->queue.empty() && (int)batch.size() < S->max_batch) {
                    uint64_t tk = S->queue.front();
                    S->queue.pop_front();
                    batch.push_back(tk);
                    items.push_back(S->reqs[tk].item);
                }
        }
        if (batch.empty()) continue;

        // 4. plan the batch; shrink it until its block fits in the arena
        BatchPlan *P = nullptr;
        size_t bytes = 0, off = 0;
        size_t n = batch.size();
        bool placed = false, build_failed = false;
        while (n > 0) {
            std::vector<const LinkDev *> devs(n);
            std::vector<drt_scene_view> views(n);
            std::vector<drt_time_grid> tgs(n);
            std::vector<drt_freq_grid> fgs(n);
            std::vector<void *> Hs(n);
            std::vector<OutD> outs(n);
            for (size_t i = 0; i < n; ++i) {
                devs[i] = &items[i].dev;
                views[i] = items[i].view;
                tgs[i] = items[i].tg;
                fgs[i] = items[i].fg;
                Hs[i] = items[i].H;
                outs[i] = items[i].out;
            }
            if (batch_build(devs, views, tgs.data(), fgs.data(), Hs.data(), outs.data(), &P, &bytes) != cudaSuccess) {
                batch_free(P);
                P = nullptr;
                build_failed = true;
                break;
            }
            {
                std::lock_guard<std::mutex> lk(S->m);
                placed = S->arena_take(bytes, &off);
            }
            if (placed) break;
            batch_free(P);
            P = nullptr;
            n = n > 1 ? n / 2 : 0;
        }
        if (build_failed) {   // the planner could not describe this batch: its requests fail
            fail_requests(S, batch, DRT_EINVAL);
            S->cv_done.notify_all();
            continue;
        }
        if (!placed) {
            // with batches in flight: back to the queue until memory frees up; with none, the
            // oldest request alone is larger than the whole arena and fails
            bool any_busy = false;
            {
                std::lock_guard<std::mutex> lk(S->m);
                for (auto &sl : S->slots) any_busy = any_busy || sl.busy;
                for (size_t i = batch.size(); i-- > (any_busy ? 0 : 1);) S->queue.push_front(batch[i]);
            }
            if (!any_busy) fail_requests(S, {batch[0]}, DRT_ENOMEM);
            S->cv_done.notify_all();
            if (any_busy) {
                std::unique_lock<std::mutex> lk(S->m);
                S->cv.wait_for(lk, std::chrono::milliseconds(5), [&] {
                    for (auto &sl : S->slots)
                        if (sl.completed) return true;
                    return S->stop;
                });
            }
            continue;
        }
        if (n < batch.size()) {   // the rest goes back to the head of the queue
            std::lock_guard<std::mutex> lk(S->m);
            for (size_t i = batch.size(); i-- > n;) S->queue.push_front(batch[i]);
            batch.resize(n);
        }

        // 5. launch on the slot's stream (no lock held across CUDA calls: the completion callback
        //    takes the lock)
        cudaError_t e = batch_bind(P, S->arena + off, slot->stream);
        const int F = items[0].fg.n_bins;
        int variant = -1;
        {
            std::lock_guard<std::mutex> lk(S->m);
            auto it = S->variant_of_bins.find(F);
            if (it != S->variant_of_bins.end()) variant = it->second;
        }
        if (e == cudaSuccess && variant < 0) {
            float ms = 0.f;
            e = batch_autotune(P, slot->stream, &ms);
            variant = batch_variant(P);
            if (e == cudaSuccess) {   // a failed tuning run is not remembered
                std::lock_guard<std::mutex> lk(S->m);
                S->variant_of_bins[F] = variant;
            }
        }
        batch_set_variant(P, variant);
        const double t_launch = now_s();
        {
            std::lock_guard<std::mutex> lk(S->m);
            slot->busy = true;
            slot->plan = P;
            slot->off = off;
            slot->size = bytes;
            slot->tickets = batch;
            for (uint64_t tk : batch) {
                Request &r = S->reqs[tk];
                r.res.t_launch = t_launch;
                r.res.batch_requests = (int32_t)batch.size();
            }
            S->stats.launches++;
        }
        if (e == cudaSuccess) e = batch_run(P, slot->stream, false);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(slot->overflow, batch_redo_overflow(P), sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, slot->stream);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(slot->stream, on_batch_done, slot);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(slot->stream);
            {
                std::lock_guard<std::mutex> lk(S->m);
                S->fatal = cudaGetErrorString(e);
                slot->completed = true;
            }
            fail_requests(S, batch, DRT_ECUDA);
            S->cv_done.notify_all();
        }
    }
}

Server *server_start(int device, void *arena, size_t arena_bytes, int n_slots, int max_batch) {
    Server *S = new Server();
    S->device = device;
    S->arena = reinterpret_cast<char *>(arena);
    S->arena_bytes = arena_bytes & ~(size_t)255;
    if (S->arena_bytes) S->free_blocks[0] = S->arena_bytes;
    S->max_batch = std::max(1, max_batch);
    S->slots.resize(std::max(1, n_slots));
    for (size_t i = 0; i < S->slots.size(); ++i) {
        S->slots[i].srv = S;
        S->slots[i].index = (int)i;
        if (cudaStreamCreateWithFlags(&S->slots[i].stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&S->slots[i].overflow), sizeof(unsigned long long),
                          cudaHostAllocDefault) != cudaSuccess) {
            for (size_t j = 0; j <= i; ++j) {
                if (S->slots[j].stream) cudaStreamDestroy(S->slots[j].stream);
                if (S->slots[j].overflow) cudaFreeHost(S->slots[j].overflow);
            }
            delete S;
            return nullptr;
        }
        *S->slots[i].overflow = 0;
    }
    S->stats.arena_bytes = S->arena_bytes;
    S->th = std::thread(serve_loop, S);
    return S;
}

// drain the queue, wait for the batches in flight, end the thread
void server_stop(Server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
    }
    S->cv.notify_all();
    S->th.join();
    for (auto &sl : S->slots) {
        cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.overflow);
    }
    delete S;
}

bool server_failed(Server *S, std::string *msg) {
    std::lock_guard<std::mutex> lk(S->m);
    if (S->fatal.empty()) return false;
    *msg = S->fatal;
    return true;
}

uint64_t server_submit(Server *S, const ServeItem &item) {
    uint64_t tk;
    {
        std::lock_guard<std::mutex> lk(S->m);
        tk = S->next_ticket++;
        Request &r = S->reqs[tk];
        r.item = item;
        r.res.status = DRT_OK;
        r.res.t_submit = now_s();
        S->queue.push_back(tk);
        S->stats.submitted++;
    }
    S->cv.notify_all();
    return tk;
}

// 1 = done (result filled, ticket retired), 0 = pending, -1 = unknown ticket
int server_poll(Server *S, uint64_t tk, drt_result *res) {
    std::lock_guard<std::mutex> lk(S->m);
    auto it = S->reqs.find(tk);
    if (it == S->reqs.end()) return -1;
    if (!it->second.done) return 0;
    if (res) *res = it->second.res;
    S->reqs.erase(it);
    return 1;
}

// 1 = done, 0 = timed out, -1 = unknown ticket
int server_wait(Server *S, uint64_t tk, uint32_t timeout_ms, drt_result *res) {
    std::unique_lock<std::mutex> lk(S->m);
    auto it = S->reqs.find(tk);
    if (it == S->reqs.end()) return -1;
    bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto j = S->reqs.find(tk);
        return j == S->reqs.end() || j->second.done;
    });
    it = S->reqs.find(tk);
    if (it == S->reqs.end()) return -1;
    if (!ok || !it->second.done) return 0;
    if (res) *res = it->second.res;
    S->reqs.erase(it);
    return 1;
}

void server_stats(Server *S, drt_serve_stats *st) {
    std::lock_guard<std::mutex> lk(S->m);
    *st = S->stats;
    st->queued = S->queue.size();
    uint64_t inflight = 0;
    for (auto &sl : S->slots)
        if (sl.busy) inflight += sl.tickets.size();
    st->in_flight = inflight;
    st->arena_bytes = S->arena_bytes;
    st->arena_used = S->arena_used;
    st->arena_peak = S->arena_peak;
}

}  // namespace drt
