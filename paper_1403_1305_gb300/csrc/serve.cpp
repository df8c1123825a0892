// Serving: a request loop over resident automata with continuous batching.
//
// ac_serve_submit copies a request's text (into device memory, or into a
// page-locked slab from which the batch's launch copies it) and queues it.
// One worker thread
// per CUDA stream takes queued requests in arrival order as long as they fit
// in the device-memory budget (and at most max_batch_items of them, waiting
// up to max_wait_us for more arrivals when the batch is small), runs them as
// one ac_scan_batch launch on its stream and completes them. Requests that
// arrive while other batches are on the GPU are admitted by the next free
// worker as memory frees up, so their work overlaps on the device.
// Completion records the latency from submission to results on the host.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "ac_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    uint32_t automaton;
    int fmt;
    uint64_t n;
    uint64_t budget_bytes;  // device memory the request is charged while in flight
    uint8_t *staged = nullptr;  // copy in device memory, or
    uint8_t *pinned = nullptr;  // copy in the page-locked slab, or
    std::vector<uint8_t> text;  // copy in ordinary host memory
    uint64_t slab_off = 0, slab_len = 0, staged_len = 0;
    Clock::time_point t_arrival;  // latency counts from here (submission, or the time the caller gave)
    const uint8_t *data() const { return staged ? staged : pinned ? pinned : text.data(); }
};

// First-fit allocator over the server's page-locked slab (16-byte granules).
struct Slab {
    uint8_t *base = nullptr;
    uint64_t size = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> length
    void init(uint8_t *b, uint64_t n) {
        base = b;
        size = n;
        free_.clear();
        if (b && n) free_[0] = n;
    }
    bool alloc(uint64_t n, uint64_t *off) {
        n = (n + 15) & ~15ull;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        n = (n + 15) & ~15ull;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Done {
    ac_result r;
    int rc;
};

}  // namespace

struct ac_server {
    std::vector<const ac_automaton *> as;
    ac_serve_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_set<uint64_t> outstanding;  // issued, not yet handed back
    uint64_t next_ticket = 1;
    uint64_t mem_in_use = 0;
    uint64_t staged_bytes = 0;  // texts waiting in device memory
    bool stopping = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    Slab slab;
    // statistics
    uint64_t submitted = 0, completed = 0, launches = 0, items_launched = 0;
    std::vector<double> latencies_ms;
};

namespace {

uint64_t charge_for(const ac_automaton *a, uint64_t n, int fmt) {
    const uint64_t bytes = fmt == AC_U8 ? n : (n + 3) / 4;
    // arena rows, match keys (and their sort and record buffers), counts
    return bytes + bytes / 8 + (bytes / 256 + 4096) * 32 + (uint64_t)a->P * 8 + (1u << 16);
}

void worker_loop(ac_server *s, int w) {
    cudaSetDevice(s->device);
    cudaStream_t st = s->streams[w];
    std::vector<Request *> batch;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (!s->pending.empty() &&
                    (s->mem_in_use == 0 || s->mem_in_use + s->pending.front()->budget_bytes <=
                                               s->opts.device_mem_budget))
                    break;
                if (s->stopping && s->pending.empty()) return;
                s->cv_work.wait(lk);
            }
            // let a small batch gather more arrivals for a moment
            if (s->opts.max_wait_us && s->pending.size() < s->opts.max_batch_items && !s->stopping) {
                const auto until = Clock::now() + std::chrono::microseconds(s->opts.max_wait_us);
                s->cv_work.wait_until(lk, until, [&] {
                    return s->stopping || s->pending.size() >= s->opts.max_batch_items;
                });
            }
            uint64_t charged = 0;
            while (!s->pending.empty() && batch.size() < s->opts.max_batch_items) {
                Request *r = s->pending.front();
                if (!batch.empty() || s->mem_in_use != 0)
                    if (s->mem_in_use + charged + r->budget_bytes > s->opts.device_mem_budget) break;
                batch.push_back(r);
                charged += r->budget_bytes;
                s->pending.pop_front();
            }
            s->mem_in_use += charged;
            s->launches++;
            s->items_launched += batch.size();
        }
        if (batch.empty()) continue;
        acgb::NvtxRange nvtx_range("ac_serve batch");
        // one launch per staging kind: device-staged texts, then host ones
        std::vector<ac_result> outs(batch.size());
        std::vector<int> rcs(batch.size(), AC_OK);
        for (int mem : {AC_DEVICE, AC_HOST}) {
            std::vector<ac_batch_item> items;
            std::vector<size_t> at;
            for (size_t i = 0; i < batch.size(); ++i)
                if ((batch[i]->staged != nullptr) == (mem == AC_DEVICE)) {
                    items.push_back(ac_batch_item{batch[i]->automaton, batch[i]->fmt, batch[i]->data(), batch[i]->n});
                    at.push_back(i);
                }
            if (items.empty()) continue;
            std::vector<ac_result> part(items.size());
            const int rc = ac_scan_batch(s->as.data(), (uint32_t)s->as.size(), items.data(), (uint32_t)items.size(),
                                         mem, 0, st, part.data());
            for (size_t j = 0; j < at.size(); ++j) {
                outs[at[j]] = part[j];
                rcs[at[j]] = rc;
            }
        }
        for (Request *r : batch)
            if (r->staged) acgb::dev_free(r->staged, st);  // after the batch's work on st
        const auto now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < batch.size(); ++i) {
                Request *r = batch[i];
                s->done[r->ticket] = Done{outs[i], rcs[i]};
                s->mem_in_use -= r->budget_bytes;
                s->staged_bytes -= r->staged_len;
                s->completed++;
                s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_arrival).count());
                if (r->pinned) s->slab.release(r->slab_off, r->slab_len);
                delete r;
            }
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

// Release a device-staged text from a thread whose current device may differ.
void free_staged(ac_server *s, uint8_t *d) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    acgb::dev_free(d, cudaStreamPerThread);
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
}

int take_result(ac_server *s, uint64_t ticket, ac_result *out) {
    auto it = s->done.find(ticket);
    const int rc = it->second.rc;
    *out = it->second.r;
    s->done.erase(it);
    s->outstanding.erase(ticket);
    if (rc != AC_OK) {
        ac_result_free(out);
        return acgb::set_error(rc, "ac_serve: request %llu failed (%s)", (unsigned long long)ticket,
                               ac_strerror(rc));
    }
    return AC_OK;
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - lo);
}

}  // namespace

using acgb::set_error;

extern "C" {

int ac_serve_create(const ac_automaton *const *as, uint32_t na, const ac_serve_opts *opts, ac_server **out) {
    if (!as || !na || !out) return set_error(AC_EINVAL, "ac_serve_create: NULL argument");
    *out = nullptr;
    for (uint32_t k = 0; k < na; ++k)
        if (!as[k] || as[k]->device < 0 || as[k]->device != as[0]->device)
            return set_error(AC_EINVAL, "ac_serve_create: automata must be built on one device");
    if (opts && opts->staging != AC_STAGE_DEVICE && opts->staging != AC_STAGE_PINNED)
        return set_error(AC_EINVAL, "ac_serve_create: unknown staging %u", opts->staging);
    ac_server *s = new (std::nothrow) ac_server();
    if (!s) return set_error(AC_ENOMEM, "ac_serve_create: host allocation");
    s->as.assign(as, as + na);
    s->device = as[0]->device;
    if (opts) s->opts = *opts;
    if (!s->opts.device_mem_budget) s->opts.device_mem_budget = 4ull << 30;
    if (!s->opts.max_batch_items) s->opts.max_batch_items = 256;
    if (!s->opts.max_queue) s->opts.max_queue = 65536;
    if (!s->opts.num_streams) s->opts.num_streams = 2;
    if (!s->opts.pinned_bytes) s->opts.pinned_bytes = 1ull << 30;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    uint8_t *slab = nullptr;
    if (cudaHostAlloc((void **)&slab, s->opts.pinned_bytes, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        slab = nullptr;  // texts then wait in ordinary host memory
    }
    s->slab.init(slab, slab ? s->opts.pinned_bytes : 0);
    for (uint32_t i = 0; i < s->opts.num_streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto x : s->streams) cudaStreamDestroy(x);
            if (s->slab.base) cudaFreeHost(s->slab.base);
            if (prev >= 0) cudaSetDevice(prev);
            delete s;
            return set_error(AC_ECUDA, "ac_serve_create: cannot create streams");
        }
        s->streams.push_back(st);
    }
    if (prev >= 0) cudaSetDevice(prev);
    for (uint32_t i = 0; i < s->opts.num_streams; ++i) s->workers.emplace_back(worker_loop, s, (int)i);
    *out = s;
    return AC_OK;
}

static int submit(ac_server *s, uint32_t automaton, const uint8_t *text, uint64_t n, int fmt, uint64_t *ticket,
                  Clock::time_point arrival);

int ac_serve_submit(ac_server *s, uint32_t automaton, const uint8_t *text, uint64_t n, int fmt, uint64_t *ticket) {
    return submit(s, automaton, text, n, fmt, ticket, Clock::now());
}

int ac_serve_submit_at(ac_server *s, uint32_t automaton, const uint8_t *text, uint64_t n, int fmt,
                       uint64_t arrival_ns, uint64_t *ticket) {
    // steady_clock counts CLOCK_MONOTONIC nanoseconds on this platform
    const Clock::time_point at{std::chrono::duration_cast<Clock::duration>(std::chrono::nanoseconds(arrival_ns))};
    return submit(s, automaton, text, n, fmt, ticket, at);
}

static int submit(ac_server *s, uint32_t automaton, const uint8_t *text, uint64_t n, int fmt, uint64_t *ticket,
                  Clock::time_point arrival) {
    acgb::NvtxRange nvtx_range("ac_serve_submit");
    if (!s || !ticket || (!text && n)) return set_error(AC_EINVAL, "ac_serve_submit: NULL argument");
    if (automaton >= s->as.size()) return set_error(AC_EINVAL, "ac_serve_submit: no automaton %u", automaton);
    if (fmt != AC_U8 && fmt != AC_PACKED2) return set_error(AC_EINVAL, "ac_serve_submit: unknown format");
    if (fmt == AC_PACKED2 && s->as[automaton]->sigma != 4)
        return set_error(AC_EINVAL, "ac_serve_submit: packed text needs a 4-letter alphabet");
    if (n >= (1ull << 32)) return set_error(AC_ERANGE, "ac_serve_submit: text of 2^32 symbols or more");
    const uint64_t charge = charge_for(s->as[automaton], n, fmt);
    if (charge > s->opts.device_mem_budget)
        return set_error(AC_ERANGE, "ac_serve_submit: the text alone exceeds the device memory budget");
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(AC_ENOMEM, "ac_serve_submit: host allocation");
    r->automaton = automaton;
    r->fmt = fmt;
    r->n = n;
    r->budget_bytes = charge;
    r->t_arrival = arrival;
    const uint64_t nbytes = fmt == AC_U8 ? n : (n + 3) / 4;
    bool to_device = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->pending.size() >= s->opts.max_queue) {
            delete r;
            return set_error(AC_EBUSY, "ac_serve_submit: queue full (%u requests)", s->opts.max_queue);
        }
        if (nbytes && s->opts.staging == AC_STAGE_DEVICE && s->staged_bytes + nbytes <= s->opts.device_mem_budget) {
            s->staged_bytes += nbytes;  // reserved; returned below if the copy cannot be made
            r->staged_len = nbytes;
            to_device = true;
        } else if (nbytes && s->slab.alloc(nbytes, &r->slab_off)) {
            r->pinned = s->slab.base + r->slab_off;
            r->slab_len = nbytes;
        }
    }
    if (to_device) {
        // the copy ends before submit returns, so the caller may reuse text at once
        int prev = -1;
        cudaGetDevice(&prev);
        bool ok = prev == s->device || cudaSetDevice(s->device) == cudaSuccess;
        uint8_t *d = ok ? (uint8_t *)acgb::dev_alloc(nbytes, cudaStreamPerThread) : nullptr;
        ok = d && cudaMemcpyAsync(d, text, nbytes, cudaMemcpyHostToDevice, cudaStreamPerThread) == cudaSuccess &&
             cudaStreamSynchronize(cudaStreamPerThread) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            if (d) acgb::dev_free(d, cudaStreamPerThread);
            d = nullptr;
        }
        if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
        if (d) {
            r->staged = d;
        } else {  // no device memory at the moment: wait in host memory instead
            std::lock_guard<std::mutex> lk(s->mu);
            s->staged_bytes -= nbytes;
            r->staged_len = 0;
            if (s->slab.alloc(nbytes, &r->slab_off)) {
                r->pinned = s->slab.base + r->slab_off;
                r->slab_len = nbytes;
            }
        }
    }
    if (r->pinned) {
        memcpy(r->pinned, text, nbytes);  // outside the lock: the range is ours
    } else if (!r->staged) {
        try {
            r->text.assign(text, text + nbytes);
        } catch (...) {
            delete r;
            return set_error(AC_ENOMEM, "ac_serve_submit: host copy of the text");
        }
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping || s->pending.size() >= s->opts.max_queue) {
            const bool stopping = s->stopping;
            if (r->pinned) s->slab.release(r->slab_off, r->slab_len);
            if (r->staged) {
                free_staged(s, r->staged);
                s->staged_bytes -= r->staged_len;
            }
            delete r;
            return stopping ? set_error(AC_EINVAL, "ac_serve_submit: server is stopping")
                            : set_error(AC_EBUSY, "ac_serve_submit: queue full (%u requests)", s->opts.max_queue);
        }
        r->ticket = s->next_ticket++;
        s->outstanding.insert(r->ticket);
        s->pending.push_back(r);
        s->submitted++;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return AC_OK;
}

int ac_serve_poll(ac_server *s, uint64_t ticket, ac_result *out) {
    if (!s || !out) return set_error(AC_EINVAL, "ac_serve_poll: NULL argument");
    memset(out, 0, sizeof(*out));
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->outstanding.count(ticket)) return set_error(AC_EINVAL, "ac_serve_poll: unknown ticket");
    if (!s->done.count(ticket)) return AC_EAGAIN;
    return take_result(s, ticket, out);
}

int ac_serve_wait(ac_server *s, uint64_t ticket, uint32_t timeout_ms, ac_result *out) {
    if (!s || !out) return set_error(AC_EINVAL, "ac_serve_wait: NULL argument");
    memset(out, 0, sizeof(*out));
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->outstanding.count(ticket)) return set_error(AC_EINVAL, "ac_serve_wait: unknown ticket");
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return s->done.count(ticket) > 0; }))
        return set_error(AC_ETIMEDOUT, "ac_serve_wait: request %llu not done after %u ms",
                         (unsigned long long)ticket, timeout_ms);
    return take_result(s, ticket, out);
}

int ac_serve_stats(ac_server *s, ac_serve_stats_t *o) {
    if (!s || !o) return set_error(AC_EINVAL, "ac_serve_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->launches = s->launches;
    o->items_launched = s->items_launched;
    o->queued = s->pending.size();
    o->in_flight = s->outstanding.size() - s->done.size() - s->pending.size();
    o->p50_ms = percentile(s->latencies_ms, 0.50);
    o->p99_ms = percentile(s->latencies_ms, 0.99);
    o->mean_batch_items = s->launches ? (double)s->items_launched / s->launches : 0.0;
    return AC_OK;
}

void ac_serve_destroy(ac_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->slab.base) cudaFreeHost(s->slab.base);
    if (prev >= 0) cudaSetDevice(prev);
    for (auto &kv : s->done) ac_result_free(&kv.second.r);
    delete s;
}

}  // extern "C"
