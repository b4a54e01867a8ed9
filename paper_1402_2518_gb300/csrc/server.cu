// Serving: continuous batching of unmixing requests (include/linmin.h,
// "Serving").  Pixels are independent (the per-pixel problem of Sec. 2.2),
// so a request is cut into chunks of at most chunk_pixels pixels and the
// chunks of all requests are run, oldest request first, by `slots` worker
// threads, each with its own CUDA stream: chunks of different requests
// overlap on the device, a request that arrives while others run starts as
// soon as a slot and device memory are free, and a small request does not
// wait behind a large one's tail.
//
// Device memory: every worker keeps the handles (library copy, per-sigma
// factors, per-pixel scratch reserved for one chunk) of the libraries it
// served, so a library seen again needs no new allocation.  The bytes of
// all handles stay within hbm_budget_bytes: a worker that needs a new handle
// first destroys idle handles (least recently used first) and otherwise
// waits until a running chunk ends.  Each chunk's results are bit-identical
// to those of a linmin_unmix call over the whole cube (no per-pixel
// computation depends on the other pixels of its launch).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "api_internal.h"
#include "linmin.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Library {
    uint64_t key = 0;                // content hash with L, P (probed past collisions)
    int L = 0, P = 0;
    std::vector<float> host;         // checked copy (P x L)
    std::chrono::steady_clock::time_point last;   // last submit that used it
};

// Libraries kept by a server beyond those in use: the least recently used
// unreferenced ones (and the idle worker handles made from them) are
// dropped above this count.
constexpr size_t kMaxLibraries = 64;
constexpr uint64_t kHostIoKey = 0x9e3779b97f4a7c15ULL;   // worker-handle key of host-buffer requests

struct Request {
    long long ticket = 0;
    linmin_request r{};
    std::shared_ptr<Library> lib;
    bool host_io = false;            // some buffer is host memory
    long long chunk = 0;             // pixels per chunk for this request
    long long next = 0;              // first pixel not yet handed out
    long long done_pixels = 0;
    int running = 0;                 // chunks in flight
    linmin_status status = LINMIN_OK;
    std::string err;
    Clock::time_point t_submit, t_done;
    bool finished = false;
};

struct Entry {                       // a worker's handle for one library
    linmin_handle h = nullptr;
    size_t bytes = 0;
    long long cap = 0;               // pixels its scratch is reserved for
    bool busy = false;
    bool tune = false;               // run the autotuner on its first chunk
    Clock::time_point last;
};

struct Worker;

}  // namespace

struct linmin_server_s {
    linmin_server_options opt{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    long long next_ticket = 1;
    std::deque<std::shared_ptr<Request>> queue;          // not finished yet, FIFO
    std::map<long long, std::shared_ptr<Request>> all;   // by ticket until waited on
    std::map<uint64_t, std::shared_ptr<Library>> libs;
    std::vector<std::unique_ptr<Worker>> workers;
    size_t bytes = 0;                // device bytes of all handles
    linmin_server_stats st{};
    std::string err;
};

namespace {

struct Worker {
    linmin_server_s *s = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    std::map<uint64_t, Entry> handles;   // by library key (mixed with host_io)
    std::thread th;
};

// Autotuned lanes per pixel by (device, L, P), shared by every server of
// the process (the choice depends on the GPU and the shape only): 0 while
// one handle is being tuned (the others use the default table meanwhile).
std::mutex g_lanes_mu;
std::map<std::tuple<int, int, int>, int> g_lanes;

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ULL)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ULL; }
    return h;
}

bool is_host(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return true; }
    return !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
}

int severity(linmin_status st)
{
    return st == LINMIN_OK ? 0 : (st == LINMIN_ERR_NOT_CONVERGED ? 1 : 2);
}

// Destroy idle handles (least recently used first, any worker) until
// `need` more bytes fit in the budget.  Caller holds s->mu.
bool make_room(linmin_server_s *s, size_t need)
{
    while (s->bytes + need > s->opt.hbm_budget_bytes) {
        Worker *wv = nullptr;
        uint64_t kv = 0;
        Clock::time_point oldest = Clock::time_point::max();
        for (auto &w : s->workers)
            for (auto &kvp : w->handles)
                if (!kvp.second.busy && kvp.second.last < oldest) {
                    oldest = kvp.second.last; wv = w.get(); kv = kvp.first;
                }
        if (!wv) return false;
        Entry e = wv->handles[kv];
        wv->handles.erase(kv);
        s->bytes -= e.bytes;
        ++s->st.evictions;
        lm::destroy_async(e.h);   // ordered after that worker's queued work: no wait
    }
    return true;
}

// Keep at most kMaxLibraries libraries: drop the least recently used ones
// that no request holds and for which no worker handle is busy, with the
// idle worker handles made from them (a later library may reuse the key).
// Caller holds s->mu.
void evict_libraries(linmin_server_s *s)
{
    while (s->libs.size() > kMaxLibraries) {
        auto victim = s->libs.end();
        for (auto it = s->libs.begin(); it != s->libs.end(); ++it) {
            if (it->second.use_count() > 1) continue;            // a request holds it
            bool busy = false;
            for (auto &w : s->workers)
                for (uint64_t k : {it->first, it->first ^ kHostIoKey}) {
                    auto h = w->handles.find(k);
                    if (h != w->handles.end() && h->second.busy) busy = true;
                }
            if (busy) continue;
            if (victim == s->libs.end() || it->second->last < victim->second->last) victim = it;
        }
        if (victim == s->libs.end()) return;                      // all in use
        for (auto &w : s->workers)
            for (uint64_t k : {victim->first, victim->first ^ kHostIoKey}) {
                auto h = w->handles.find(k);
                if (h == w->handles.end()) continue;
                s->bytes -= h->second.bytes;
                ++s->st.evictions;
                lm::destroy_async(h->second.h);
                w->handles.erase(h);
            }
        s->libs.erase(victim);
    }
}

// Mark a request finished and wake its waiters.  Caller holds s->mu.
void finish(linmin_server_s *s, Request *rq)
{
    rq->finished = true;
    rq->t_done = Clock::now();
    ++s->st.requests_done;
    s->cv_done.notify_all();
}

// Next chunk to run: the oldest request with pixels not handed out whose
// handle this worker has or can get within the budget.  Caller holds s->mu.
// Returns false when nothing can run now.
bool take_chunk(Worker *w, std::shared_ptr<Request> *req, long long *first, long long *n,
                Entry **entry, uint64_t *hkey)
{
    linmin_server_s *s = w->s;
    for (size_t qi = 0; qi < s->queue.size();) {
        std::shared_ptr<Request> rq = s->queue[qi];
        if (rq->next >= rq->r.N) { ++qi; continue; }       // all chunks handed out
        const uint64_t key = rq->lib->key ^ (rq->host_io ? kHostIoKey : 0);
        auto it = w->handles.find(key);
        if (it != w->handles.end() && it->second.cap < rq->chunk) {
            // a cached handle with a smaller reservation: grow it within the budget
            Entry &e = it->second;
            const size_t need = lm::handle_bytes(rq->r.L, rq->r.P, rq->chunk, rq->host_io);
            e.busy = true;                                  // not a candidate for eviction
            const bool room = make_room(s, need - e.bytes);
            e.busy = false;
            if (!room) return false;
            if (lm::reserve(e.h, rq->chunk, rq->host_io) != LINMIN_OK) {
                s->bytes -= e.bytes;
                linmin_destroy(e.h);
                w->handles.erase(it);
                it = w->handles.end();                      // start over with a new handle
            } else {
                s->bytes += need - e.bytes;
                s->st.peak_bytes = std::max<unsigned long long>(s->st.peak_bytes, s->bytes);
                e.bytes = need;
                e.cap = rq->chunk;
            }
        }
        if (it == w->handles.end()) {
            const size_t need = lm::handle_bytes(rq->r.L, rq->r.P, rq->chunk, rq->host_io);
            if (!make_room(s, need)) return false;        // keep FIFO order: wait
            linmin_options o;
            linmin_default_options(&o);
            o.max_iter = s->opt.max_iter;
            o.cuda_stream = w->stream;
            Entry e;
            linmin_status st = lm::create_from_host(rq->lib->host.data(), rq->r.L, rq->r.P, o,
                                                    &e.h);
            if (st != LINMIN_OK) rq->err = linmin_last_error(nullptr);
            if (st == LINMIN_OK && (st = lm::reserve(e.h, rq->chunk, rq->host_io)) != LINMIN_OK)
                rq->err = linmin_last_error(e.h);
            if (st != LINMIN_OK) {
                if (e.h) linmin_destroy(e.h);
                rq->status = st;
                rq->next = rq->r.N;                          // no more chunks
                if (rq->running == 0) {
                    finish(s, rq.get());
                    s->queue.erase(s->queue.begin() + qi);
                    continue;
                }
                ++qi;
                continue;
            }
            if (s->opt.autotune) {
                std::lock_guard<std::mutex> g(g_lanes_mu);
                auto lt = g_lanes.find({s->device, rq->r.L, rq->r.P});
                if (lt == g_lanes.end()) {                   // first of its shape: tune it
                    g_lanes[{s->device, rq->r.L, rq->r.P}] = 0;
                    e.tune = true;
                } else if (lt->second > 0) {
                    linmin_set_lanes(e.h, lt->second);
                }
            }
            e.bytes = need;
            e.cap = rq->chunk;
            s->bytes += need;
            s->st.peak_bytes = std::max<unsigned long long>(s->st.peak_bytes, s->bytes);
            ++s->st.handles_created;
            it = w->handles.emplace(key, e).first;
        }
        *req = rq;
        *first = rq->next;
        *n = std::min(rq->chunk, rq->r.N - rq->next);
        rq->next += *n;
        ++rq->running;
        *entry = &it->second;
        *hkey = key;
        it->second.busy = true;
        return true;
    }
    return false;
}

void run_worker(Worker *w)
{
    linmin_server_s *s = w->s;
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        std::shared_ptr<Request> rq;
        long long first = 0, n = 0;
        Entry *e = nullptr;
        uint64_t key = 0;
        while (!s->stop && !take_chunk(w, &rq, &first, &n, &e, &key))
            s->cv_work.wait(lk);
        if (s->stop) return;
        ++s->st.running;
        s->st.max_running = std::max(s->st.max_running, s->st.running);
        linmin_handle h = e->h;
        const bool tune = e->tune;
        e->tune = false;
        lk.unlock();

        const linmin_request &r = rq->r;
        const size_t P = r.P, L = r.L, f = (size_t)first;
        if (tune) {
            // the autotuner on this chunk's pixels (synchronous, on the
            // worker's stream, outside the lock); its choice serves every
            // later handle of the shape
            int lanes = 0;
            const bool ok =
                linmin_autotune(h, r.cube + f * L, n, r.sigma, &lanes, nullptr, 0, nullptr) ==
                LINMIN_OK;
            {
                std::lock_guard<std::mutex> g(g_lanes_mu);
                if (ok) g_lanes[{s->device, r.L, r.P}] = lanes;
                else g_lanes.erase({s->device, r.L, r.P});   // a later handle tries again
            }
            if (ok) {
                std::lock_guard<std::mutex> g(s->mu);
                ++s->st.autotuned;
            }
        }
        linmin_status st = linmin_unmix(
            h, r.cube + f * L, n, r.sigma, r.abundances ? r.abundances + f * P : nullptr,
            r.uncertainties ? r.uncertainties + f * P : nullptr,
            r.residual_rms ? r.residual_rms + f : nullptr, r.iterations ? r.iterations + f : nullptr);
        if (st == LINMIN_OK || st == LINMIN_ERR_NOT_CONVERGED) {
            const linmin_status sw = linmin_wait(h, nullptr);   // device buffers: wait here
            if (severity(sw) > severity(st)) st = sw;
        }
        std::string why = st == LINMIN_OK ? std::string() : std::string(linmin_last_error(h));

        lk.lock();
        --s->st.running;
        ++s->st.chunks;
        auto it = w->handles.find(key);
        if (it != w->handles.end()) { it->second.busy = false; it->second.last = Clock::now(); }
        --rq->running;
        rq->done_pixels += n;
        if (severity(st) > severity(rq->status)) { rq->status = st; rq->err = why; }
        if (severity(st) == 2) rq->next = r.N;             // stop handing out chunks
        if (rq->running == 0 && rq->next >= r.N) {
            finish(s, rq.get());
            s->queue.erase(std::find(s->queue.begin(), s->queue.end(), rq));
        }
        s->cv_work.notify_all();                            // memory or a slot was freed
    }
}

linmin_status sfail(linmin_server s, linmin_status st, const std::string &m)
{
    if (s) { std::lock_guard<std::mutex> g(s->mu); s->err = m; }
    return st;
}

}  // namespace

extern "C" {

linmin_status linmin_server_default_options(linmin_server_options *opt)
{
    if (!opt) return LINMIN_ERR_INVALID;
    opt->hbm_budget_bytes = 1ULL << 30;
    opt->slots = 4;
    opt->chunk_pixels = 65536;
    opt->max_iter = 100;
    opt->autotune = 1;
    return LINMIN_OK;
}

linmin_status linmin_server_create(const linmin_server_options *opt, linmin_server *out)
{
    if (!out) return LINMIN_ERR_INVALID;
    *out = nullptr;
    linmin_server_options o;
    linmin_server_default_options(&o);
    if (opt) o = *opt;
    if (o.slots < 1 || o.slots > 64 || o.chunk_pixels < 1 || o.max_iter < 1 ||
        o.hbm_budget_bytes == 0)
        return LINMIN_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return LINMIN_ERR_CUDA; }
    linmin_server_s *s = new linmin_server_s();
    s->opt = o;
    s->device = dev;
    for (int i = 0; i < o.slots; ++i) {
        auto w = std::make_unique<Worker>();
        w->s = s;
        w->index = i;
        if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s->workers.push_back(std::move(w));
            linmin_server_destroy(s);
            return LINMIN_ERR_CUDA;
        }
        s->workers.push_back(std::move(w));
    }
    for (auto &w : s->workers) w->th = std::thread(run_worker, w.get());
    *out = s;
    return LINMIN_OK;
}

linmin_status linmin_server_submit(linmin_server s, const linmin_request *req, long long *ticket)
{
    if (!s || !req || !ticket) return LINMIN_ERR_INVALID;
    *ticket = 0;
    const linmin_request &r = *req;
    if (r.P < 1 || r.P > LINMIN_MAX_P)
        return sfail(s, LINMIN_ERR_UNSUPPORTED, "P must be in [1, LINMIN_MAX_P]");
    if (r.L < r.P || r.L > LINMIN_MAX_L) return sfail(s, LINMIN_ERR_INVALID, "L must be in [P, 4096]");
    if (!r.library || !r.sigma || (r.N > 0 && !r.cube) || r.N < 0)
        return sfail(s, LINMIN_ERR_INVALID, "library, sigma and cube are required, N >= 0");

    auto rq = std::make_shared<Request>();
    rq->r = r;
    rq->t_submit = Clock::now();
    rq->host_io = is_host(r.cube) || is_host(r.sigma) || is_host(r.abundances) ||
                  is_host(r.uncertainties) || is_host(r.residual_rms) || is_host(r.iterations);
    // the library: content hash, checked once per distinct library
    std::vector<float> host;
    std::string why;
    const linmin_status lst = lm::load_library(r.library, r.L, r.P, &host, &why);
    if (lst != LINMIN_OK) return sfail(s, lst, why);
    uint64_t key = fnv1a(host.data(), host.size() * 4);
    key = fnv1a(&r.L, sizeof r.L, key);
    key = fnv1a(&r.P, sizeof r.P, key);
    // pixels per chunk: at most chunk_pixels, and one handle must fit the budget
    long long chunk = std::max<long long>(1, std::min<long long>(s->opt.chunk_pixels, r.N));
    while (chunk > 1 && lm::handle_bytes(r.L, r.P, chunk, rq->host_io) > s->opt.hbm_budget_bytes)
        chunk /= 2;
    if (lm::handle_bytes(r.L, r.P, chunk, rq->host_io) > s->opt.hbm_budget_bytes)
        return sfail(s, LINMIN_ERR_OOM, "one chunk of this request exceeds hbm_budget_bytes");
    rq->chunk = chunk;

    std::lock_guard<std::mutex> g(s->mu);
    // a hit must hold the same library, not only the same hash: on a
    // collision, probe the next key
    auto li = s->libs.find(key);
    while (li != s->libs.end() &&
           !(li->second->L == r.L && li->second->P == r.P && li->second->host == host))
        li = s->libs.find(++key);
    if (li == s->libs.end()) {
        auto lib = std::make_shared<Library>();
        lib->key = key; lib->L = r.L; lib->P = r.P; lib->host = std::move(host);
        li = s->libs.emplace(key, lib).first;
    }
    li->second->last = Clock::now();
    rq->lib = li->second;
    evict_libraries(s);
    s->st.libraries = (long long)s->libs.size();
    rq->ticket = s->next_ticket++;
    *ticket = rq->ticket;
    s->all[rq->ticket] = rq;
    ++s->st.requests;
    if (r.N == 0) {
        finish(s, rq.get());
        return LINMIN_OK;
    }
    s->queue.push_back(rq);
    s->cv_work.notify_all();
    return LINMIN_OK;
}

linmin_status linmin_server_poll(linmin_server s, long long ticket, int *done)
{
    if (!s || !done) return LINMIN_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return LINMIN_ERR_INVALID;
    *done = it->second->finished ? 1 : 0;
    return LINMIN_OK;
}

linmin_status linmin_server_wait(linmin_server s, long long ticket, double *latency_ms)
{
    if (!s) return LINMIN_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) { s->err = "unknown ticket"; return LINMIN_ERR_INVALID; }
    std::shared_ptr<Request> rq = it->second;
    s->cv_done.wait(lk, [&] { return rq->finished; });
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count();
    s->all.erase(ticket);
    if (rq->status != LINMIN_OK) s->err = rq->err;
    return rq->status;
}

linmin_status linmin_server_get_stats(linmin_server s, linmin_server_stats *st)
{
    if (!s || !st) return LINMIN_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    *st = s->st;
    st->bytes = s->bytes;
    return LINMIN_OK;
}

unsigned long long linmin_server_handle_bytes(int L, int P, long long chunk_pixels, int host_io)
{
    if (P < 1 || P > LINMIN_MAX_P || L < P || L > LINMIN_MAX_L || chunk_pixels < 0) return 0;
    return lm::handle_bytes(L, P, chunk_pixels, host_io != 0);
}

const char *linmin_server_last_error(linmin_server s)
{
    static thread_local std::string msg;
    if (!s) return "server is NULL";
    std::lock_guard<std::mutex> g(s->mu);
    msg = s->err;
    return msg.c_str();
}

linmin_status linmin_server_destroy(linmin_server s)
{
    if (!s) return LINMIN_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // let the requests already submitted finish
        s->cv_done.wait(lk, [&] { return s->queue.empty(); });
        s->stop = true;
        s->cv_work.notify_all();
    }
    for (auto &w : s->workers)
        if (w->th.joinable()) w->th.join();
    for (auto &w : s->workers) {
        for (auto &kv : w->handles) linmin_destroy(kv.second.h);
        if (w->stream) cudaStreamDestroy(w->stream);
    }
    delete s;
    return LINMIN_OK;
}

}  // extern "C"
