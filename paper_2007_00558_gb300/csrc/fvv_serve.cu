// fvv_serve.cu -- continuous-batching serving loop over the view-synthesis
// path.
//
// Many viewers each request their own virtual viewpoint (the paper's
// interactive use: a viewer moves the virtual camera and waits for the new
// view, Sec. VIII motion-to-photon delay).  Requests of any resolution are
// admitted into a queue; a scheduler thread packs them, in arrival order,
// into batched launches of steps a-e on `lanes` CUDA streams.  Each lane owns
// device scratch sized from the memory budget, so a batch is admitted only
// when a lane and its memory are free, and batches on different lanes overlap
// on the GPU.  Requests that arrive while batches run join the next batch as
// soon as a lane frees up (continuous batching).  Every batch renders from
// the newest complete frame tick at the moment it is formed.  An event
// recorded after each batch's last work is polled by a completion thread,
// which stamps each request's completion; latency is submission to
// completion of its output write.
//
// With refinement on, a lane renders its batch (all requests of one size)
// into its own device buffers of network inputs (colour, depth, hole mask,
// top-3 weights); the network then runs on one refinement stream shared by
// the lanes, ordered after the plain batch by an event, writes the refined
// colour into the lane and copies each request's view out.  The plain pass
// of one lane overlaps the network pass of another.  The network's
// activations are sized once, at start, for the largest batch a lane holds.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "fvv_runtime.h"

namespace fvv {

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum class ReqState { Queued, Running, Done, Failed };

struct Req {
    uint64_t ticket;
    uint32_t viewer;
    fvv_view view;
    uint8_t* out;
    size_t pitch;
};

struct Rec {
    ReqState state = ReqState::Queued;
    double t_submit = 0.0;
    double t_done = 0.0;
};

}  // namespace

struct ServeLane {
    ServeState* owner = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    BatchScratch S;
    bool busy = false;
    std::vector<uint64_t> tickets;
    // refinement: network inputs and refined colour for `px` pixels, one
    // allocation of kRefineBytesPerPixel * px bytes
    uint8_t* feat = nullptr;
    size_t px = 0;
    float *depth = nullptr, *top3 = nullptr;
    uint8_t *rgb = nullptr, *hole = nullptr, *refined = nullptr;
    cudaEvent_t plain_done = nullptr;
    int* flag_host = nullptr;             // pinned copy of the network's error flag
    cudaEvent_t done_ev = nullptr;        // recorded after a batch's last work (stream lanes)
    bool ev_pending = false;              // done_ev recorded, its requests not yet completed
};

struct ServeState {
    fvv_ctx* ctx = nullptr;
    fvv_serve_cfg cfg{};
    std::thread thread;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> queue;
    std::unordered_map<uint64_t, Rec> recs;
    std::vector<std::unique_ptr<ServeLane>> lanes;
    size_t lane_keys = 0, lane_stage = 0;
    cudaStream_t refine_stream = nullptr;
    bool reset_flag = false;              // a batch saw the network's error flag raised
    bool stopping = false;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batch_views = 0;
    std::vector<double> lat_ms;
    double t_first = -1.0, t_last = -1.0;
    std::string error;
    // persistent mode: the batch ring (pinned, mapped), its device alias, the
    // kernel's barrier state, its stream and an event recorded after its
    // launch (complete once it returned), and the poller thread
    PersistQueue* pq = nullptr;
    PersistQueue* pq_dev = nullptr;
    PersistSync* psync = nullptr;
    cudaStream_t pstream = nullptr;
    cudaEvent_t pexit = nullptr;
    bool plaunched = false;
    int pctas = 0;
    uint32_t pposted = 0;                  // batches posted (host's count; pq->posted mirrors it)
    ServeLane* pslot[kPersistRing] = {};   // the lane of posted batch b at b % kPersistRing
    std::thread poller;
    bool poller_stop = false;
    // stream lanes: the thread that polls the lanes' done events
    std::thread completer;
    bool completer_stop = false;
};

namespace {

// network inputs (depth 4 + top-3 weights 12 + colour 3 + hole 1) and the
// refined colour (3), bytes per pixel of a lane
constexpr size_t kRefineBytesPerPixel = 23;

// persistent mode: a grid barrier of the kernel gives up after 2 s
constexpr uint64_t kPersistBarrierNs = 2000000000ull;

// Whether the persistent kernel is (still) running; caller holds c->mu.
bool persist_running(ServeState* st)
{
    if (!st->plaunched) return false;
    const cudaError_t e = cudaEventQuery(st->pexit);
    if (e == cudaErrorNotReady) return true;
    if (e != cudaSuccess) cudaGetLastError();
    return false;
}

// Launch the persistent kernel for the batches from pq->done on, unless it
// runs; caller holds c->mu.
fvv_status persist_launch(fvv_ctx* c, ServeState* st)
{
    if (persist_running(st)) return FVV_OK;
    st->plaunched = false;
    FVV_CUDA(cudaMemsetAsync(st->psync, 0, sizeof(PersistSync), st->pstream));
    st->pq->err = 0;
    int ctas = 0;
    // the other CTAs wait at a grid barrier while CTA 0 waits for work: the
    // barrier's limit stays above the idle limit
    const uint64_t idle_ns = uint64_t(st->cfg.idle_us) * 1000ull;
    const uint64_t wait_ns = std::max<uint64_t>(kPersistBarrierNs, idle_ns + 1000000000ull);
    const cudaError_t e = launch_serve_persistent(st->pq_dev, st->psync, st->pq->done, st->cfg.max_width, c->n_cams,
                                                  idle_ns, wait_ns, st->pstream, &ctas);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FVV_ERR_CUDA, std::string("persistent serving kernel: ") + cudaGetErrorString(e));
    }
    FVV_CUDA(cudaEventRecord(st->pexit, st->pstream));
    st->plaunched = true;
    return FVV_OK;
}

// Batches [from, to) completed at time t (ok) or failed; caller holds st->mu.
void persist_finish(ServeState* st, uint32_t from, uint32_t to, double t, bool ok)
{
    for (uint32_t b = from; b < to; ++b) {
        ServeLane* L = st->pslot[b % kPersistRing];
        st->pslot[b % kPersistRing] = nullptr;
        if (!L) continue;
        for (uint64_t tk : L->tickets) {
            auto it = st->recs.find(tk);
            if (it == st->recs.end()) continue;
            if (!ok) {
                it->second.state = ReqState::Failed;
                ++st->failed;
                continue;
            }
            it->second.state = ReqState::Done;
            it->second.t_done = t;
            st->lat_ms.push_back(1e3 * (t - it->second.t_submit));
            ++st->completed;
        }
        L->tickets.clear();
        L->busy = false;
    }
    if (ok) st->t_last = t;
}

// Poller: publishes the batches the kernel completed (their requests Done,
// their lanes free), and relaunches the kernel when it returned (idle) with
// batches still posted, or fails those batches when it returned because a
// wait ran out.
void persist_poller(ServeState* st)
{
    fvv_ctx* c = st->ctx;
    cudaSetDevice(c->device);
    uint32_t seen = st->pq->done;
    // whether the kernel still runs is asked only after 100 us without
    // progress, and never waits for the context lock (an upload may hold
    // it): the completion count alone answers the common case
    double t_progress = now_s();
    for (;;) {
        const uint32_t d = st->pq->done;
        if (d != seen) {
            const double t = now_s();
            {
                std::lock_guard<std::mutex> lk(st->mu);
                persist_finish(st, seen, d, t, true);
            }
            st->cv.notify_all();
            seen = d;
            t_progress = t;
            continue;
        }
        uint32_t posted;
        {
            std::lock_guard<std::mutex> lk(st->mu);
            if (st->poller_stop) break;
            posted = st->pposted;
        }
        if (posted == d) t_progress = now_s();
        if (posted != d && now_s() - t_progress > 1e-4) {
            std::unique_lock<std::recursive_mutex> g(c->mu, std::try_to_lock);
            if (!g.owns_lock()) {
                std::this_thread::yield();
                continue;
            }
            t_progress = now_s();
            if (!persist_running(st) && st->pq->done == d) {
                if (st->pq->err != 0) {
                    // a wait of the kernel ran out: its pending batches fail
                    {
                        std::lock_guard<std::mutex> lk(st->mu);
                        st->error = "a bounded wait of the persistent serving kernel ran out (code " +
                                    std::to_string(st->pq->err) + ")";
                        persist_finish(st, d, posted, now_s(), false);
                    }
                    st->pq->done = posted;
                    seen = posted;
                    st->cv.notify_all();
                } else if (persist_launch(c, st) != FVV_OK) {
                    std::lock_guard<std::mutex> lk(st->mu);
                    st->error = fvv_last_error();
                    persist_finish(st, d, posted, now_s(), false);
                    st->pq->done = posted;
                    seen = posted;
                    st->cv.notify_all();
                }
            }
        }
        // a batch outstanding: poll again at once (latency); idle: sleep
        if (posted != st->pq->done)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Complete lane L's batch at time t (its work has finished, or failed with
// `cuda_err`); caller holds st->mu.
void lane_finish(ServeState* st, ServeLane* L, double t, cudaError_t cuda_err)
{
    {
        const bool timed_out = cuda_err == cudaSuccess && L->flag_host && *L->flag_host != 0;
        if (cuda_err != cudaSuccess) {
            st->error = std::string("a serving batch failed: ") + cudaGetErrorString(cuda_err);
            for (uint64_t tk : L->tickets) {
                auto it = st->recs.find(tk);
                if (it == st->recs.end()) continue;
                it->second.state = ReqState::Failed;
                ++st->failed;
            }
            L->tickets.clear();
            L->busy = false;
            return;
        }
        if (timed_out) {
            st->reset_flag = true;
            st->error = "a bounded wait of the refinement network ran out";
        }
        for (uint64_t tk : L->tickets) {
            auto it = st->recs.find(tk);
            if (it == st->recs.end()) continue;
            if (timed_out) {
                it->second.state = ReqState::Failed;
                ++st->failed;
                continue;
            }
            it->second.state = ReqState::Done;
            it->second.t_done = t;
            st->lat_ms.push_back(1e3 * (t - it->second.t_submit));
            ++st->completed;
        }
        st->t_last = t;
        L->tickets.clear();
        L->busy = false;
    }
}

// Stream lanes: completes a lane's requests as soon as its done event is
// reached.  It polls (yielding) while any batch is in flight and sleeps on
// the condition variable otherwise, which answers faster than a host
// callback enqueued on the stream.
void lane_completer(ServeState* st)
{
    cudaSetDevice(st->ctx->device);
    std::unique_lock<std::mutex> lk(st->mu);
    for (;;) {
        bool any = false;
        for (auto& Lp : st->lanes) {
            ServeLane* L = Lp.get();
            if (!L->ev_pending) continue;
            any = true;
            lk.unlock();
            const cudaError_t q = cudaEventQuery(L->done_ev);
            lk.lock();
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            L->ev_pending = false;
            lane_finish(st, L, now_s(), q);
            st->cv.notify_all();
        }
        if (!any) {
            if (st->completer_stop) break;
            st->cv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
    }
}

// One refined batch of same-size views on lane L: plain steps a-e into the
// lane's network inputs on the lane's stream, then, on the refinement
// stream, the network into the lane's refined colour, each request's copy
// out and a copy of the network's error flag.  The caller holds c->mu.
fvv_status run_refined(fvv_ctx* c, ServeState* st, ServeLane* L, const std::vector<fvv_view>& views,
                       const std::vector<Req>& reqs, std::vector<fvv_aux>& aux, std::vector<uint8_t*>& outs,
                       std::vector<size_t>& pitches)
{
    const int n = int(views.size()), W = views[0].width, H = views[0].height;
    const size_t np = size_t(W) * H;
    aux.assign(n, fvv_aux{});
    for (int i = 0; i < n; ++i) {
        outs[i] = L->rgb + size_t(i) * np * 3;
        pitches[i] = size_t(W) * 3;
        aux[i].depth = L->depth + size_t(i) * np;
        aux[i].hole = L->hole + size_t(i) * np;
        aux[i].top3 = L->top3 + size_t(i) * np * 3;
    }
    FVV_TRY(run_batch(c, L->S, n, views.data(), nullptr, outs.data(), pitches.data(), aux.data(), L->stream,
                      false));
    FVV_CUDA(cudaEventRecord(L->plain_done, L->stream));
    FVV_CUDA(cudaStreamWaitEvent(st->refine_stream, L->plain_done, 0));
    fvv_refine_batch b{};
    b.n = n;
    b.height = H;
    b.width = W;
    b.rgb = L->rgb;
    b.depth = L->depth;
    b.hole = L->hole;
    b.top3 = L->top3;
    FVV_TRY(refine_forward_async(c, b, L->refined, st->refine_stream));
    for (int i = 0; i < n; ++i)
        FVV_CUDA(cudaMemcpy2DAsync(reqs[i].out, reqs[i].pitch, L->refined + size_t(i) * np * 3, size_t(W) * 3,
                                   size_t(W) * 3, size_t(H), cudaMemcpyDefault, st->refine_stream));
    int* flag = nullptr;
    FVV_TRY(refine_error_flag(&flag));
    FVV_CUDA(cudaMemcpyAsync(L->flag_host, flag, sizeof(int), cudaMemcpyDeviceToHost, st->refine_stream));
    return FVV_OK;
}

// Persistent mode: prepare the batch (parameters copied, waits for the
// frames' uploads queued on the lane's stream), wait for that on the host,
// then post it to the kernel's ring and make sure the kernel runs.  Its
// completion comes through the poller.
fvv_status persist_submit(fvv_ctx* c, ServeState* st, ServeLane* L, const std::vector<fvv_view>& views,
                          std::vector<uint8_t*>& outs, std::vector<size_t>& pitches)
{
    PersistPost P;
    P.ctas = st->pctas;
    {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        FVV_TRY(run_batch(c, L->S, int(views.size()), views.data(), nullptr, outs.data(), pitches.data(), nullptr,
                          L->stream, false, &P));
        FVV_CUDA(cudaEventRecord(L->plain_done, L->stream));
    }
    FVV_CUDA(cudaEventSynchronize(L->plain_done));
    std::lock_guard<std::recursive_mutex> g(c->mu);
    uint32_t b;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        b = st->pposted;
        st->pslot[b % kPersistRing] = L;
    }
    st->pq->batch[b % kPersistRing] = P.batch;
    for (int si : P.slots) c->slot[si].persist_reads = b + 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);      // the batch before its index
    st->pq->posted = b + 1;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->pposted = b + 1;
    }
    return persist_launch(c, st);
}

void scheduler(ServeState* st)
{
    fvv_ctx* c = st->ctx;
    cudaSetDevice(c->device);
    std::vector<fvv_view> views;
    std::vector<uint8_t*> outs;
    std::vector<size_t> pitches;
    std::vector<Req> reqs;
    std::vector<fvv_aux> aux;
    std::unique_lock<std::mutex> lk(st->mu);
    for (;;) {
        auto free_lane = [&]() -> ServeLane* {
            for (auto& L : st->lanes)
                if (!L->busy) return L.get();
            return nullptr;
        };
        auto idle = [&]() {
            for (auto& L : st->lanes)
                if (L->busy) return false;
            return true;
        };
        st->cv.wait_for(lk, std::chrono::milliseconds(5), [&] {
            return (st->stopping && st->queue.empty() && idle()) ||
                   (!st->queue.empty() && free_lane() != nullptr);
        });
        if (st->stopping && st->queue.empty() && idle()) break;
        // coalescing window: a short queue waits for its oldest request to
        // age batch_window_us (stopping sends it at once)
        if (st->cfg.batch_window_us && !st->stopping && !st->queue.empty() &&
            int(st->queue.size()) < st->cfg.max_batch) {
            const double due = st->recs[st->queue.front().ticket].t_submit + 1e-6 * st->cfg.batch_window_us;
            const double wait = due - now_s();
            if (wait > 0.0) {
                st->cv.wait_for(lk, std::chrono::duration<double>(wait),
                                [&] { return st->stopping || int(st->queue.size()) >= st->cfg.max_batch; });
                continue;
            }
        }
        if (st->reset_flag) {
            // a network wait ran out: clear the flag before the next batch
            st->reset_flag = false;
            lk.unlock();
            int* flag = nullptr;
            {
                std::lock_guard<std::recursive_mutex> g(c->mu);
                if (refine_error_flag(&flag) == FVV_OK)
                    cudaMemsetAsync(flag, 0, sizeof(int), st->refine_stream);
            }
            lk.lock();
        }
        ServeLane* L;
        while (!st->queue.empty() && (L = free_lane()) != nullptr) {
            views.clear();
            outs.clear();
            pitches.clear();
            reqs.clear();
            L->tickets.clear();
            auto take = [&](const Req& r) {
                views.push_back(r.view);
                outs.push_back(r.out);
                pitches.push_back(r.pitch);
                reqs.push_back(r);
                L->tickets.push_back(r.ticket);
                st->recs[r.ticket].state = ReqState::Running;
            };
            if (st->cfg.refine) {
                // the oldest request and later ones of its size, up to the
                // lane's pixels (one network batch is one size)
                const int W = st->queue.front().view.width, H = st->queue.front().view.height;
                const size_t np = size_t(W) * H;
                size_t px = 0;
                for (auto it = st->queue.begin();
                     it != st->queue.end() && int(views.size()) < st->cfg.max_batch;) {
                    if (it->view.width == W && it->view.height == H && px + np <= L->px) {
                        px += np;
                        take(*it);
                        it = st->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            } else {
                // the oldest requests that fit this lane's scratch
                size_t keys = 0, stage = 0;
                while (!st->queue.empty() && int(views.size()) < st->cfg.max_batch) {
                    const Req& r = st->queue.front();
                    const size_t k = view_keys(r.view, c->opt.layered != 0),
                                 b = view_stage_bytes(r.view, r.out, nullptr);
                    if (keys + k > L->S.keys_cap || stage + b > L->S.out_stage_cap) break;
                    keys += k;
                    stage += b;
                    take(r);
                    st->queue.pop_front();
                }
            }
            L->busy = true;
            ++st->batches;
            st->batch_views += views.size();
            lk.unlock();
            fvv_status rc;
            std::string err;
            if (st->cfg.persistent) {
                rc = persist_submit(c, st, L, views, outs, pitches);
                if (rc != FVV_OK) err = fvv_last_error();
            } else {
                std::lock_guard<std::recursive_mutex> g(c->mu);
                cudaStream_t done_on = L->stream;
                if (st->cfg.refine) {
                    rc = run_refined(c, st, L, views, reqs, aux, outs, pitches);
                    done_on = st->refine_stream;
                } else {
                    rc = run_batch(c, L->S, int(views.size()), views.data(), nullptr, outs.data(),
                                   pitches.data(), nullptr, L->stream, false);
                }
                if (rc == FVV_OK) {
                    cudaError_t e = cudaEventRecord(L->done_ev, done_on);
                    if (e != cudaSuccess) {
                        cudaGetLastError();
                        rc = FVV_ERR_CUDA;
                        err = std::string("cudaEventRecord: ") + cudaGetErrorString(e);
                    }
                } else {
                    err = fvv_last_error();
                }
                if (rc != FVV_OK) {
                    // work of this batch may be queued: let it drain before
                    // the lane's buffers are reused
                    cudaStreamSynchronize(L->stream);
                    if (st->refine_stream) cudaStreamSynchronize(st->refine_stream);
                }
            }
            lk.lock();
            if (rc == FVV_OK && !st->cfg.persistent) {
                L->ev_pending = true;              // the completer takes it from here
                st->cv.notify_all();
            }
            if (rc != FVV_OK) {
                for (uint64_t tk : L->tickets) {
                    st->recs[tk].state = ReqState::Failed;
                    ++st->failed;
                }
                L->tickets.clear();
                L->busy = false;
                st->error = err;
                st->cv.notify_all();
            }
        }
    }
}

// Release a lane's stream, scratch and refinement buffers (work drained).
void lane_free(fvv_ctx* c, ServeLane& L)
{
    if (L.stream) cudaStreamSynchronize(L.stream);
    scratch_free(c, L.S);
    dev_free(c, L.feat, L.px * kRefineBytesPerPixel);
    L.feat = nullptr;
    if (L.flag_host) cudaFreeHost(L.flag_host);
    L.flag_host = nullptr;
    if (L.plain_done) cudaEventDestroy(L.plain_done);
    L.plain_done = nullptr;
    if (L.done_ev) cudaEventDestroy(L.done_ev);
    L.done_ev = nullptr;
    if (L.stream) cudaStreamDestroy(L.stream);
    L.stream = nullptr;
}

// The lane's refinement buffers for `px` pixels (a multiple of 64).
fvv_status lane_refine_alloc(fvv_ctx* c, ServeLane& L, size_t px)
{
    FVV_TRY(dev_alloc(c, reinterpret_cast<void**>(&L.feat), px * kRefineBytesPerPixel));
    L.px = px;
    L.depth = reinterpret_cast<float*>(L.feat);
    L.top3 = reinterpret_cast<float*>(L.feat + px * 4);
    L.rgb = L.feat + px * 16;
    L.refined = L.feat + px * 19;
    L.hole = L.feat + px * 22;
    FVV_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&L.flag_host), sizeof(int), cudaHostAllocDefault));
    *L.flag_host = 0;
    FVV_CUDA(cudaEventCreateWithFlags(&L.plain_done, cudaEventDisableTiming));
    return FVV_OK;
}

}  // namespace

bool serve_refining(fvv_ctx* c) { return c && c->serve && c->serve->cfg.refine; }

fvv_status serve_wait_slot(fvv_ctx* c, const SlotState& slot)
{
    ServeState* st = c->serve;
    if (!st || !st->pq || slot.persist_reads == 0) return FVV_OK;
    const double t0 = now_s();
    while (st->pq->done < slot.persist_reads) {
        if (st->pq->err == 0 && !persist_running(st)) FVV_TRY(persist_launch(c, st));   // it returned, idle
        if (now_s() - t0 > 2.0)
            return fail(FVV_ERR_TIMEOUT, "a persistent serving batch still reads this frame slot after 2 s");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    return FVV_OK;
}

void serve_shutdown(fvv_ctx* c)
{
    ServeState* st = c->serve;
    if (!st) return;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->stopping = true;
    }
    st->cv.notify_all();
    if (st->thread.joinable()) st->thread.join();
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->completer_stop = true;           // the scheduler left only when every lane was idle
    }
    st->cv.notify_all();
    if (st->completer.joinable()) st->completer.join();
    if (st->pq) {
        // every request finished; the kernel returns at its next wait for work
        st->pq->stop = 1;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        if (st->pstream) cudaStreamSynchronize(st->pstream);
        {
            std::lock_guard<std::mutex> lk(st->mu);
            st->poller_stop = true;
        }
        if (st->poller.joinable()) st->poller.join();
    }
    {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        if (st->pq) {
            for (int si = 0; si < c->slots; ++si) c->slot[si].persist_reads = 0;
            cudaFreeHost(st->pq);
            st->pq = nullptr;
            dev_free(c, st->psync, sizeof(PersistSync));
            if (st->pexit) cudaEventDestroy(st->pexit);
            if (st->pstream) cudaStreamDestroy(st->pstream);
        }
        if (st->refine_stream) cudaStreamSynchronize(st->refine_stream);
        for (auto& L : st->lanes) lane_free(c, *L);
        if (st->refine_stream) cudaStreamDestroy(st->refine_stream);
    }
    c->serve = nullptr;
    delete st;
}

}  // namespace fvv

using fvv::ReqState;
using fvv::ServeState;
using fvv::fail;

extern "C" {

fvv_status fvv_serve_default_cfg(fvv_serve_cfg* cfg)
{
    if (!cfg) return fail(FVV_ERR_INVALID_ARG, "cfg is NULL");
    cfg->lanes = 3;
    cfg->max_batch = 16;
    cfg->max_pending = 4096;
    cfg->memory_budget = uint64_t(768) << 20;
    cfg->refine = 0;
    cfg->persistent = 0;
    cfg->max_width = 1920;
    cfg->idle_us = 20000;
    cfg->batch_window_us = 0;
    return FVV_OK;
}

fvv_status fvv_serve_start(fvv_ctx* c, const fvv_serve_cfg* cfg_in)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    fvv::DeviceScope dev_scope(c->device);
    fvv_serve_cfg cfg;
    if (cfg_in) cfg = *cfg_in; else fvv_serve_default_cfg(&cfg);
    if (cfg.lanes < 1 || cfg.lanes > fvv::kMaxReaders - 1)
        return fail(FVV_ERR_INVALID_ARG, "lanes must be in [1, 16]");
    if (cfg.max_batch < 1 || cfg.max_batch > 4096 || cfg.max_pending < 1)
        return fail(FVV_ERR_INVALID_ARG, "max_batch must be in [1, 4096], max_pending >= 1");
    if (cfg.refine != 0 && cfg.refine != 1) return fail(FVV_ERR_INVALID_ARG, "refine must be 0 or 1");
    if (cfg.batch_window_us > 1000000) return fail(FVV_ERR_INVALID_ARG, "batch_window_us must be at most 1 s");
    if (cfg.persistent != 0 && cfg.persistent != 1) return fail(FVV_ERR_INVALID_ARG, "persistent must be 0 or 1");
    if (cfg.persistent) {
        if (cfg.refine) return fail(FVV_ERR_INVALID_ARG, "persistent serving renders plain views (refine = 0)");
        if (c->opt.layered) return fail(FVV_ERR_INVALID_ARG, "persistent serving needs a single-layer context");
        if (cfg.lanes > fvv::kPersistRing) return fail(FVV_ERR_INVALID_ARG, "persistent serving: at most 16 lanes");
        if (cfg.idle_us < 100 || cfg.idle_us > 10000000)
            return fail(FVV_ERR_INVALID_ARG, "idle_us must be in [100, 10000000]");
        if (cfg.max_width < 1 || fvv::resolve_smem_bytes(cfg.max_width, c->n_cams, false) > c->smem_optin)
            return fail(FVV_ERR_INVALID_ARG, "max_width must be >= 1 and fit the shared memory");
    }
    if (c->serve) return fail(FVV_ERR_STATE, "serving loop already running");
    std::lock_guard<std::recursive_mutex> g(c->mu);
    if (cfg.refine && !fvv::refine_ready(c))
        return fail(FVV_ERR_STATE, "refine = 1 needs fvv_refine_init first");
    FVV_CUDA(cudaSetDevice(c->device));
    auto st = std::make_unique<ServeState>();
    st->ctx = c;
    st->cfg = cfg;
    const size_t per_lane = size_t(cfg.memory_budget) / size_t(cfg.lanes);
    const size_t pb = fvv::align_up(size_t(cfg.max_batch) * sizeof(fvv::ViewDesc), 256) +
                      size_t(cfg.max_batch) * c->n_cams * sizeof(fvv::CamGeom);
    if (per_lane < 2 * pb + (size_t(1) << 20))
        return fail(FVV_ERR_BUDGET, "memory_budget too small for the lanes");
    const size_t room = per_lane - 2 * pb;
    size_t lane_px = 0;
    if (cfg.refine) {
        // per lane and pixel: 8 bytes of keys per z-buffer (three when
        // layered) and the refinement buffers
        const size_t layers = c->opt.layered ? 3 : 1;
        lane_px = room / (8 * layers + fvv::kRefineBytesPerPixel) / 64 * 64;
        st->lane_keys = lane_px * layers;
        st->lane_stage = 0;
    } else {
        // per lane: 8 bytes of keys and 3 bytes of host-output staging per pixel
        st->lane_keys = fvv::align_up(room / 11, 16) - 16;
        st->lane_stage = fvv::align_up((room - st->lane_keys * 8) & ~size_t(255), 256) - 256;
    }
    auto unwind = [&](fvv_status rc, const std::string& msg) {
        if (st->refine_stream) cudaStreamSynchronize(st->refine_stream);
        for (auto& l : st->lanes) fvv::lane_free(c, *l);
        if (st->refine_stream) cudaStreamDestroy(st->refine_stream);
        if (st->pexit) cudaEventDestroy(st->pexit);
        if (st->pstream) cudaStreamDestroy(st->pstream);
        return fail(rc, msg);
    };
    if (cfg.refine) {
        cudaError_t e = cudaStreamCreateWithFlags(&st->refine_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return unwind(FVV_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        // the network's activations for the largest batch a lane holds
        if (fvv::refine_reserve(c, lane_px) != FVV_OK) return unwind(FVV_ERR_BUDGET, fvv_last_error());
    }
    for (int i = 0; i < cfg.lanes; ++i) {
        auto L = std::make_unique<fvv::ServeLane>();
        L->owner = st.get();
        L->index = i;
        cudaError_t e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
        fvv_status rc = e == cudaSuccess ? FVV_OK : FVV_ERR_CUDA;
        if (rc == FVV_OK)
            rc = fvv::scratch_alloc(c, L->S, st->lane_keys, st->lane_stage, cfg.max_batch, 2);
        if (rc == FVV_OK && cfg.refine) rc = fvv::lane_refine_alloc(c, *L, lane_px);
        if (rc == FVV_OK && cfg.persistent) {
            e = cudaEventCreateWithFlags(&L->plain_done, cudaEventDisableTiming);
            if (e != cudaSuccess) rc = FVV_ERR_CUDA;
        }
        if (rc == FVV_OK) {
            e = cudaEventCreateWithFlags(&L->done_ev, cudaEventDisableTiming);
            if (e != cudaSuccess) rc = FVV_ERR_CUDA;
        }
        L->S.reader = 1 + i;
        st->lanes.push_back(std::move(L));
        if (rc != FVV_OK)
            return unwind(rc, e != cudaSuccess ? std::string("cudaStreamCreate: ") + cudaGetErrorString(e)
                                               : std::string(fvv_last_error()));
    }
    if (cfg.persistent) {
        void* q = nullptr;
        cudaError_t e = cudaHostAlloc(&q, sizeof(fvv::PersistQueue), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            std::memset(q, 0, sizeof(fvv::PersistQueue));
            st->pq = static_cast<fvv::PersistQueue*>(q);
            e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&st->pq_dev), q, 0);
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st->pstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->pexit, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (st->pq) cudaFreeHost(st->pq);
            st->pq = nullptr;
            return unwind(FVV_ERR_CUDA, std::string("persistent serving setup: ") + cudaGetErrorString(e));
        }
        void* ps = nullptr;
        if (fvv::dev_alloc(c, &ps, sizeof(fvv::PersistSync)) != FVV_OK) {
            cudaFreeHost(st->pq);
            st->pq = nullptr;
            return unwind(FVV_ERR_OUT_OF_MEMORY, fvv_last_error());
        }
        st->psync = static_cast<fvv::PersistSync*>(ps);
        st->pctas = fvv::persist_grid(cfg.max_width, c->n_cams);
        if (st->pctas < 1) {
            cudaFreeHost(st->pq);
            st->pq = nullptr;
            fvv::dev_free(c, ps, sizeof(fvv::PersistSync));
            return unwind(FVV_ERR_CUDA, "persistent serving kernel: no resident CTA fits");
        }
    }
    ServeState* raw = st.release();
    c->serve = raw;
    raw->thread = std::thread(fvv::scheduler, raw);
    if (raw->pq) raw->poller = std::thread(fvv::persist_poller, raw);
    else raw->completer = std::thread(fvv::lane_completer, raw);
    return FVV_OK;
}

fvv_status fvv_serve_submit(fvv_ctx* c, uint32_t viewer, const fvv_view* view, uint8_t* out,
                            size_t pitch, uint64_t* ticket)
{
    if (!c || !view || !out || !ticket) return fail(FVV_ERR_INVALID_ARG, "NULL argument");
    ServeState* st = c->serve;
    if (!st) return fail(FVV_ERR_STATE, "serving loop not running");
    fvv::DeviceScope dev_scope(c->device);
    if (fvv::foreign(out)) return fail(FVV_ERR_INVALID_ARG, "out must be host memory or the context's device memory");
    std::string why;
    if (!fvv::camera_ok(*view, &why)) return fail(FVV_ERR_INVALID_ARG, "view: " + why);
    if (fvv::resolve_smem_bytes(view->width, c->n_cams, c->opt.layered != 0) > c->smem_optin)
        return fail(FVV_ERR_INVALID_ARG, "view: width too large");
    if (pitch < size_t(view->width) * 3) return fail(FVV_ERR_INVALID_ARG, "pitch < 3 * width");
    if (st->cfg.persistent) {
        if (view->width > st->cfg.max_width)
            return fail(FVV_ERR_INVALID_ARG, "view wider than the persistent kernel's max_width");
        if (fvv::mem_kind(out) != fvv::MemKind::Device)
            return fail(FVV_ERR_INVALID_ARG, "persistent serving writes device outputs only");
    }
    if (st->cfg.refine) {
        if (view->width % 4 || view->height % 4)
            return fail(FVV_ERR_INVALID_ARG, "refined views need width and height multiples of 4");
        if (size_t(view->width) * view->height > st->lanes[0]->px)
            return fail(FVV_ERR_BUDGET, "view does not fit one lane's share of the serving memory budget");
    } else if (fvv::view_keys(*view, c->opt.layered != 0) > st->lane_keys ||
               fvv::view_stage_bytes(*view, out, nullptr) > st->lane_stage) {
        return fail(FVV_ERR_BUDGET, "view does not fit one lane's share of the serving memory budget");
    }
    {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        if (!c->have_any) return fail(FVV_ERR_NOT_READY, "no frame uploaded yet");
    }
    {
        std::lock_guard<std::mutex> lk(st->mu);
        if (st->stopping) return fail(FVV_ERR_STATE, "serving loop is stopping");
        if (st->recs.size() >= size_t(st->cfg.max_pending))
            return fail(FVV_ERR_BUSY, "max_pending requests outstanding; poll some first");
        const uint64_t t = st->next_ticket++;
        fvv::Rec r;
        r.t_submit = fvv::now_s();
        st->recs.emplace(t, r);
        st->queue.push_back(fvv::Req{t, viewer, *view, out, pitch});
        ++st->submitted;
        if (st->t_first < 0.0) st->t_first = r.t_submit;
        *ticket = t;
    }
    st->cv.notify_all();
    return FVV_OK;
}

fvv_status fvv_serve_poll(fvv_ctx* c, uint64_t ticket, int64_t timeout_us)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    ServeState* st = c->serve;
    if (!st) return fail(FVV_ERR_STATE, "serving loop not running");
    std::unique_lock<std::mutex> lk(st->mu);
    auto it = st->recs.find(ticket);
    if (it == st->recs.end()) return fail(FVV_ERR_INVALID_ARG, "unknown or already collected ticket");
    auto finished = [&] {
        auto i = st->recs.find(ticket);
        return i->second.state == ReqState::Done || i->second.state == ReqState::Failed;
    };
    if (!finished()) {
        if (timeout_us == 0) return fail(FVV_ERR_NOT_READY, "request not finished");
        if (timeout_us < 0)
            st->cv.wait(lk, finished);
        else if (!st->cv.wait_for(lk, std::chrono::microseconds(timeout_us), finished))
            return fail(FVV_ERR_TIMEOUT, "request not finished within the timeout");
    }
    it = st->recs.find(ticket);
    const bool ok = it->second.state == ReqState::Done;
    st->recs.erase(it);
    if (!ok) return fail(FVV_ERR_CUDA, "request failed: " + st->error);
    return FVV_OK;
}

fvv_status fvv_serve_stats(fvv_ctx* c, fvv_serve_report* out, int32_t reset)
{
    if (!c || !out) return fail(FVV_ERR_INVALID_ARG, "NULL argument");
    ServeState* st = c->serve;
    if (!st) return fail(FVV_ERR_STATE, "serving loop not running");
    std::lock_guard<std::mutex> lk(st->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = st->submitted;
    out->completed = st->completed;
    out->failed = st->failed;
    out->batches = st->batches;
    out->mean_batch = st->batches ? double(st->batch_views) / double(st->batches) : 0.0;
    int running = 0;
    for (auto& kv : st->recs)
        if (kv.second.state == ReqState::Queued || kv.second.state == ReqState::Running) ++running;
    out->in_flight = running;
    if (!st->lat_ms.empty()) {
        std::vector<double> v = st->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const size_t i = size_t(std::ceil(q * double(v.size()))) - 1;
            return v[std::min(i, v.size() - 1)];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
    }
    if (st->completed && st->t_last > st->t_first)
        out->views_per_s = double(st->completed) / (st->t_last - st->t_first);
    if (reset) {
        st->submitted = st->completed = st->failed = st->batches = st->batch_views = 0;
        st->lat_ms.clear();
        st->t_first = st->t_last = -1.0;
    }
    return FVV_OK;
}

fvv_status fvv_serve_stop(fvv_ctx* c)
{
    if (!c) return fail(FVV_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->serve) return fail(FVV_ERR_STATE, "serving loop not running");
    fvv::DeviceScope dev_scope(c->device);
    fvv::serve_shutdown(c);
    return FVV_OK;
}

}  // extern "C"
