// Continuous-batching request loop over a batch (smre_server_* of
// include/smre.h).
//
// Callers submit projection requests from any thread; a loop thread owns the
// batch.  Each round it admits waiting requests in arrival order while a slot
// and enough arena bytes (the request's increment-storage footprint) are
// free, enqueues a few cycles for every admitted image, then retires the
// images that stopped (copying their results out) so their slots and bytes
// admit the next requests.  Requests that arrive while others are on the GPU
// join at the next round, and their cycles share the launches of the others.
// Because an image's arithmetic does not depend on the other images in the
// batch, a result is the same whatever else was being served.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "smre_internal.h"

using namespace smre;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    long long ticket = 0;
    int H = 0, W = 0;
    std::vector<float> x0;     // the caller's image, copied at submission
    float *out = nullptr;      // caller's result buffer (host or device)
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    smre_result res{};
    smre_status status = SMRE_OK;
    bool done = false;
};

}  // namespace

struct smre_server {
    smre_batch *b = nullptr;
    size_t arena_bytes = 0;
    smre_batch_params bp{};
    std::vector<int> sides;
    std::vector<double> cexp;
    int device = 0;
    int cycles_per_round = 4;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;                  // arrival order
    std::map<int, Request *> by_slot;               // admitted, on the GPU
    std::unordered_map<long long, std::unique_ptr<Request>> all;
    long long next_ticket = 1;
    bool stop = false;
    std::thread loop;
    // statistics
    std::vector<double> latency;                    // submit -> result, completed requests
    long long submitted = 0, completed = 0, rounds = 0;
    int peak_active = 0;
    double t_first = 0.0, t_last = 0.0;
    smre_status loop_status = SMRE_OK;
    std::string err;
};

namespace {

void finish(smre_server *s, Request *r, smre_status st)
{
    std::lock_guard<std::mutex> lk(s->mu);
    r->status = st;
    r->done = true;
    r->t_done = now_s();
    s->latency.push_back(r->t_done - r->t_submit);
    ++s->completed;
    s->t_last = r->t_done;
    s->cv_done.notify_all();
}

void run_loop(smre_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty() || !s->by_slot.empty(); });
            if (s->stop && s->pending.empty() && s->by_slot.empty()) return;
        }
        // admission, in arrival order, while a slot and the arena have room
        for (;;) {
            Request *r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->pending.empty()) break;
                r = s->pending.front();
            }
            int slot = -1;
            const smre_status st = smre_batch_submit(s->b, r->H, r->W, r->x0.data(), &slot);
            if (st != SMRE_OK) {
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->pending.pop_front();
                }
                finish(s, r, st);
                continue;
            }
            if (slot < 0) break;   // full: wait for retirements
            std::lock_guard<std::mutex> lk(s->mu);
            s->pending.pop_front();
            r->t_admit = now_s();
            s->by_slot[slot] = r;
            s->peak_active = std::max(s->peak_active, (int)s->by_slot.size());
            std::vector<float>().swap(r->x0);   // the batch holds its own copy now
        }
        bool any;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            any = !s->by_slot.empty();
        }
        if (!any) continue;
        smre_status st = smre_batch_run(s->b, s->cycles_per_round);
        std::vector<int> done(s->bp.max_images);
        int n = 0;
        if (st == SMRE_OK) st = smre_batch_poll(s->b, done.data(), (int)done.size(), &n);
        ++s->rounds;
        if (st != SMRE_OK) {
            // a failed round fails every image on the GPU; the batch stays usable
            std::vector<std::pair<int, Request *>> lost;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                lost.assign(s->by_slot.begin(), s->by_slot.end());
                s->by_slot.clear();
                s->loop_status = st;
                s->err = smre_batch_last_error(s->b);
            }
            for (auto &pr : lost) {
                batch_drop(s->b, pr.first);
                finish(s, pr.second, st);
            }
            continue;
        }
        for (int k = 0; k < n; ++k) {
            Request *r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r = s->by_slot[done[k]];
                s->by_slot.erase(done[k]);
            }
            const smre_status rs = smre_batch_retrieve(s->b, done[k], r->out, &r->res);
            finish(s, r, rs);
        }
    }
}

}  // namespace

extern "C" {

smre_status smre_server_create(const smre_server_params *p, void *cuda_stream, smre_server **out)
{
    const AllocScope scope;
    if (!out || !p) {
        set_thread_error("params / out is NULL");
        return SMRE_EINVAL;
    }
    *out = nullptr;
    if (p->cycles_per_round < 1) {
        set_thread_error("cycles_per_round must be >= 1");
        return SMRE_EINVAL;
    }
    smre_server *s = new (std::nothrow) smre_server;
    if (!s) return SMRE_ENOMEM;
    s->bp = p->batch;
    s->sides.assign(p->batch.sides, p->batch.sides + std::max(p->batch.n_sides, 0));
    if (p->batch.c_explicit)
        s->cexp.assign(p->batch.c_explicit, p->batch.c_explicit + std::max(p->batch.n_sides, 0));
    s->bp.sides = s->sides.data();
    s->bp.c_explicit = p->batch.c_explicit ? s->cexp.data() : nullptr;
    s->cycles_per_round = p->cycles_per_round;
    cudaGetDevice(&s->device);
    const smre_status st = smre_batch_create(&s->bp, cuda_stream, &s->b);
    if (st != SMRE_OK) {
        delete s;
        return st;
    }
    s->arena_bytes = p->batch.device_bytes;
    s->loop = std::thread(run_loop, s);
    *out = s;
    return SMRE_OK;
}

smre_status smre_server_submit(smre_server *s, int height, int width, const float *x0, float *x,
                               long long *ticket)
{
    if (!s || !x0 || !x || !ticket) {
        set_thread_error("server / x0 / x / ticket is NULL");
        return SMRE_EINVAL;
    }
    const size_t need = smre_batch_image_bytes(&s->bp, height, width);
    if (need == 0) {
        set_thread_error("image size not supported by the server's batch");
        return SMRE_EINVAL;
    }
    if (need > s->arena_bytes) {
        set_thread_error("image needs more device bytes than the server's arena holds");
        return SMRE_EINVAL;
    }
    auto r = std::make_unique<Request>();
    r->H = height;
    r->W = width;
    r->out = x;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, x0) == cudaSuccess && at.type == cudaMemoryTypeDevice) {
        r->x0.resize((size_t)height * width);
        if (cudaMemcpy(r->x0.data(), x0, sizeof(float) * r->x0.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            set_thread_error("copy of a device x0 failed");
            return SMRE_ECUDA;
        }
    } else {
        cudaGetLastError();
        r->x0.assign(x0, x0 + (size_t)height * width);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->t_submit = now_s();
    if (s->submitted == 0) s->t_first = r->t_submit;
    ++s->submitted;
    *ticket = r->ticket;
    s->pending.push_back(r.get());
    s->all[r->ticket] = std::move(r);
    s->cv_work.notify_one();
    return SMRE_OK;
}

smre_status smre_server_wait(smre_server *s, long long ticket, double timeout_s, smre_result *res)
{
    if (!s) return SMRE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_thread_error("unknown ticket");
        return SMRE_EINVAL;
    }
    Request *r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return SMRE_ETIMEOUT;   // not finished yet; the ticket stays valid
    }
    if (res) {
        *res = r->res;
        res->seconds = r->t_done - r->t_submit;
    }
    const smre_status st = r->status;
    s->all.erase(it);
    return st;
}

smre_status smre_server_stats(smre_server *s, smre_server_counters *out)
{
    if (!s || !out) return SMRE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->waiting = (int)s->pending.size();
    out->active = (int)s->by_slot.size();
    out->peak_active = s->peak_active;
    out->rounds = s->rounds;
    if (!s->latency.empty()) {
        std::vector<double> l = s->latency;
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
        out->p50_s = q(0.50);
        out->p99_s = q(0.99);
        out->max_s = l.back();
        double m = 0.0;
        for (double v : l) m += v;
        out->mean_s = m / l.size();
    }
    if (s->completed > 0 && s->t_last > s->t_first)
        out->images_per_s = s->completed / (s->t_last - s->t_first);
    return s->loop_status;
}

void smre_server_destroy(smre_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;   // the loop drains what was submitted, then ends
        s->cv_work.notify_all();
    }
    if (s->loop.joinable()) s->loop.join();
    smre_batch_destroy(s->b);
    delete s;
}

}  // extern "C"
