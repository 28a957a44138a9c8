// Serving: a request loop with continuous batching, built on the batch-slot,
// count, enumerate and length entry points of the C ABI.
//
// Requests (count, length range with an optional histogram, enumerate) are
// queued by fs_server_submit.  One worker thread admits them into reusable
// batch slots, each with its own stream: a slot takes whatever has arrived (up
// to max_batch queries) as soon as it is free, so requests that arrive while
// other batches are on the GPU are batched and run concurrently with them.
// Per-query planning state and slice queues stay on the device inside the
// slot.  The batch counts every request; an enumerate (its rows) or a length
// histogram then becomes a job, admitted in arrival order when its exact
// output bytes fit the server's device memory budget (refused with
// FS_E_CAPACITY when they exceed the whole budget) and one of the job streams
// is idle, so several jobs run at once beside the batches.  A count or length
// request whose walk is long skips the batch and is a job from the start
// (direct): the single-query walk takes it with the whole GPU, and the
// batch's other answers do not wait for it.  Completed requests are collected
// by fs_server_poll with a timestamp per stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/fs.h"
#include "launch.h"

namespace {

struct Req {
    uint64_t ticket;
    fs_request r;
    double t_submit;
    double t_start;    // its batch was launched
    double t_counted;  // its batch's results were collected
    double t_job;      // its job was launched (0: none)
    bool direct;       // COUNT / LENGTHS run as a job of its own (no batch)
};

struct Slot {
    fs_batch* b = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Req> reqs;
    std::vector<fs_result> res;
};

// Device work after the batch: an enumerate's rows or a length histogram.
struct Job {
    Req req;
    uint64_t count;
    uint32_t min_len, max_len;
    uint64_t off, bytes;  // output in the pool
    bool refuse_hist;     // direct LENGTHS whose histogram is over the work bound
    // whether the job holds pool memory: all but the direct ones without a histogram
    bool pooled() const { return !req.direct || bytes > 0; }
};

struct JobLane {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    uint64_t* dscratch = nullptr;  // device counters the job writes (count, min, max)
    uint64_t* hres = nullptr;      // pinned copy of them, for direct jobs
    bool busy = false;
    Job job;
};

// First-fit allocator over the server's row budget.
struct Pool {
    char* base = nullptr;
    uint64_t size = 0;
    std::map<uint64_t, uint64_t> free_blocks;  // offset -> size
    bool alloc(uint64_t bytes, uint64_t* off)
    {
        bytes = (bytes + 255) & ~(uint64_t)255;
        if (bytes == 0) bytes = 256;
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes;
                const uint64_t o = it->first + bytes;
                free_blocks.erase(it);
                if (rest) free_blocks[o] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        bytes = (bytes + 255) & ~(uint64_t)255;
        if (bytes == 0) bytes = 256;
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

}  // namespace

struct fs_server {
    fs_server_config cfg;
    int dev = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_in, cv_done;
    std::deque<Req> pending;
    std::deque<fs_response> done;
    std::map<uint64_t, std::pair<uint64_t, uint64_t>> held;  // ticket -> (off, bytes)
    bool stop = false;
    uint64_t next_ticket = 1;
    std::thread worker;
    std::vector<Slot> slots;
    std::vector<JobLane> lanes;
    Pool pool;
    std::deque<Job> job_wait;
    fs_status fatal = FS_OK;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    void finish(const Req& q, int32_t status, uint64_t count, uint32_t mn, uint32_t mx, void* rows)
    {
        fs_response r;
        memset(&r, 0, sizeof r);
        r.ticket = q.ticket;
        r.status = status;
        r.op = q.r.op;
        r.count = count;
        r.min_len = mn;
        r.max_len = mx;
        r.rows = rows;
        r.t_submit = q.t_submit;
        r.t_start = q.t_start;
        r.t_counted = q.t_counted;
        r.t_job = q.t_job;
        r.t_done = now();
        std::lock_guard<std::mutex> lk(mu);
        done.push_back(r);
        cv_done.notify_all();
    }

    bool busy_gpu() const
    {
        for (const Slot& o : slots)
            if (o.busy) return true;
        for (const JobLane& l : lanes)
            if (l.busy) return true;
        return false;
    }

    bool step();
    void run();
};

// The smallest generator of a request (its longest length is n / min g).
static uint32_t min_gen(const fs_request& r)
{
    uint32_t m = 0xffffffffu;
    for (int i = 0; i < r.d && i < FS_MAX_D; i++) m = std::min(m, r.gens[i]);
    return m;
}

// Leaves the PAIR length walk of a request visits: prefixes of the first d-2
// generators (descending) whose residual the gcd G of the last two divides,
// i.e. the factorizations of n over those d-2 generators and G.  Exact by a
// DP over 0..n (floating point, enough for a threshold) while n <= 2^20, else
// the leading term n^(k-1) / ((k-1)! prod g) of that count (k = d - 1
// generators).
static double hist_walk_leaves(const fs_request& r)
{
    std::vector<uint64_t> g(r.gens, r.gens + std::min(r.d, (int32_t)FS_MAX_D));
    std::sort(g.begin(), g.end(), std::greater<uint64_t>());
    if (g.size() < 3) return 1.0;
    uint64_t a = g[g.size() - 1], b = g[g.size() - 2];
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    g.resize(g.size() - 2);
    g.push_back(a);
    const uint64_t n = (uint64_t)std::max<int64_t>(r.n, 0);
    if (n <= (1u << 20)) {
        std::vector<double> f(n + 1, 0.0);
        f[0] = 1.0;
        for (uint64_t h : g)
            for (uint64_t p = h; p <= n; p++) f[p] += f[p - h];
        return f[n];
    }
    double v = 1.0 / (double)g.back();
    for (size_t i = 0; i + 1 < g.size(); i++) v *= (double)n / (double)g[i] / (double)(i + 1);
    return v;
}

// Leaves the batched walk of a request visits, estimated from above by the
// lattice volume: the walk takes the generators in descending order, all but
// the last four (d >= 5 and n < 2^22), three (d >= 4) or two, and the prefixes
// with sum a_i g_i <= n number at most prod_i (n + S) / ((i + 1) g_i) (S the
// sum of those generators).  0 for a request the batch rejects anyway.
static double batch_walk_leaves(const fs_request& r)
{
    if (r.d < 1 || r.d > FS_MAX_D || r.n < 0) return 0.0;
    std::vector<double> g(r.gens, r.gens + r.d);
    for (double x : g)
        if (x < 1.0) return 0.0;
    std::sort(g.begin(), g.end(), std::greater<double>());
    const int k = (r.d >= 5 && r.n < (1 << 22)) ? 4 : (r.d >= 4 && r.n < (1 << 27)) ? 3 : 2;
    const int m = std::max(0, r.d - k);
    double S = 0.0;
    for (int i = 0; i < m; i++) S += g[i];
    double v = 1.0;
    for (int i = 0; i < m; i++) v *= ((double)r.n + S) / ((double)(i + 1) * g[i]);
    return v;
}

bool fs_server::step()
{
    bool progress = false;
    // 1. finished batches: answer the requests, or queue their jobs
    for (Slot& sl : slots) {
        if (!sl.busy || cudaEventQuery(sl.ev) != cudaSuccess) continue;
        sl.res.resize(sl.reqs.size());
        fs_status s = fs_batch_collect(sl.b, sl.res.data());
        const double tc = now();
        for (size_t i = 0; i < sl.reqs.size(); i++) {
            Req& q = sl.reqs[i];
            q.t_counted = tc;
            const fs_result& R = sl.res[i];
            const int32_t st = s != FS_OK ? s : R.status;
            const bool enum_job = q.r.op == FS_REQ_ENUMERATE;
            const bool hist_job = q.r.op == FS_REQ_LENGTHS && q.r.hist;
            if (hist_job && st == FS_OK && hist_walk_leaves(q.r) > (double)cfg.hist_max_leaves) {
                finish(q, FS_E_CAPACITY, R.count, R.min_len, R.max_len, nullptr);
            } else if ((enum_job || hist_job) && st == FS_OK) {
                Job j;
                j.req = q;
                j.count = R.count;
                j.min_len = R.min_len;
                j.max_len = R.max_len;
                j.off = 0;
                j.bytes = enum_job ? R.count * (uint64_t)q.r.d * (uint64_t)q.r.elem_bytes
                                   : ((uint64_t)q.r.n / min_gen(q.r) + 1) * 8;
                j.refuse_hist = false;
                job_wait.push_back(j);
            } else {
                finish(q, st, R.count, R.min_len, R.max_len, nullptr);
            }
        }
        sl.reqs.clear();
        sl.busy = false;
        progress = true;
    }
    // 2. finished jobs: their outputs stay reserved until released; a direct
    // job's count (and length range) comes from its own walk
    for (JobLane& l : lanes) {
        if (!l.busy || cudaEventQuery(l.ev) != cudaSuccess) continue;
        Job& j = l.job;
        if (j.req.direct) {
            j.req.t_counted = now();
            j.count = l.hres[0];
            if (j.req.r.op == FS_REQ_LENGTHS) {
                j.min_len = (uint32_t)l.hres[1];
                j.max_len = (uint32_t)l.hres[2];
            }
        }
        if (!j.pooled()) {
            finish(j.req, j.refuse_hist ? FS_E_CAPACITY : FS_OK, j.count, j.min_len, j.max_len, nullptr);
        } else {
            {
                std::lock_guard<std::mutex> lk(mu);
                held[j.req.ticket] = {j.off, j.bytes};
            }
            finish(j.req, FS_OK, j.count, j.min_len, j.max_len, pool.base + j.off);
        }
        l.busy = false;
        progress = true;
    }
    // 3. start jobs in arrival order, each admitted by its exact output bytes
    for (JobLane& l : lanes) {
        if (l.busy) continue;
        bool started = false;
        while (!started && !job_wait.empty()) {
            Job& j = job_wait.front();
            if (j.bytes > pool.size) {
                finish(j.req, FS_E_CAPACITY, j.count, j.min_len, j.max_len, nullptr);
                job_wait.pop_front();
                progress = true;
                continue;
            }
            bool ok = true;
            if (j.pooled()) {
                std::lock_guard<std::mutex> lk(mu);
                ok = pool.alloc(j.bytes, &j.off);
            }
            if (!ok) break;  // wait for outputs to be released
            j.req.t_job = now();
            if (j.req.direct) j.req.t_start = j.req.t_job;
            fs_config ec;
            fs_config_default(&ec);
            fs_status s;
            uint64_t* hist = j.pooled() ? (uint64_t*)(pool.base + j.off) : nullptr;
            if (j.req.r.op == FS_REQ_ENUMERATE) {
                ec.keep_order = j.req.r.keep_order;
                s = fs_enumerate_async(j.req.r.n, j.req.r.gens, j.req.r.d, &ec, pool.base + j.off,
                                       j.count, j.req.r.elem_bytes, l.dscratch, l.st);
            } else if (j.req.r.op == FS_REQ_COUNT) {
                s = fs_count_async(j.req.r.n, j.req.r.gens, j.req.r.d, &ec, l.dscratch, l.st);
            } else {
                s = fs_length_stats_async(j.req.r.n, j.req.r.gens, j.req.r.d, &ec, hist, l.dscratch,
                                          l.st);
            }
            if (s == FS_OK && j.req.direct &&
                cudaMemcpyAsync(l.hres, l.dscratch, 3 * 8, cudaMemcpyDeviceToHost, l.st) != cudaSuccess)
                s = FS_E_CUDA;
            if (s != FS_OK) {
                if (j.pooled()) {
                    std::lock_guard<std::mutex> lk(mu);
                    pool.release(j.off, j.bytes);
                }
                finish(j.req, s, j.count, j.min_len, j.max_len, nullptr);
                job_wait.pop_front();
                progress = true;
                continue;
            }
            cudaEventRecord(l.ev, l.st);
            l.job = j;
            l.busy = true;
            job_wait.pop_front();
            started = progress = true;
        }
        if (job_wait.empty()) break;
    }
    // 3b. long count / length requests become jobs of their own, in arrival
    // order behind the jobs already waiting
    {
        std::vector<Req> direct;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (auto it = pending.begin(); it != pending.end();) {
                if (it->direct) {
                    direct.push_back(*it);
                    it = pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        for (const Req& q : direct) {
            Job j;
            j.req = q;
            j.count = 0;
            j.min_len = j.max_len = 0;
            j.off = 0;
            j.bytes = 0;
            j.refuse_hist = false;
            if (q.r.op == FS_REQ_LENGTHS && q.r.hist) {
                // a histogram over the work bound or larger than the whole budget:
                // count and range only, then FS_E_CAPACITY
                const uint64_t hb = ((uint64_t)q.r.n / min_gen(q.r) + 1) * 8;
                if (hist_walk_leaves(q.r) > (double)cfg.hist_max_leaves || hb > pool.size)
                    j.refuse_hist = true;
                else
                    j.bytes = hb;
            }
            job_wait.push_back(j);
            progress = true;
        }
    }
    // 4. admit arrived requests into a free slot.  A batch holds one class of
    // requests, that of the oldest one waiting: counts alone (count mode, no
    // length tables) or the rest (lengths mode: count and length range); each
    // class keeps its arrival order.
    for (Slot& sl : slots) {
        if (sl.busy) continue;
        std::vector<Req> take;
        int mode = FS_BATCH_LENGTHS;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (pending.empty()) break;
            // while other work is on the GPU, let the batch fill for up to
            // window_us; an idle GPU takes what has arrived at once
            const bool gpu_busy = busy_gpu();
            const double age = now() - pending.front().t_submit;
            if (gpu_busy && (int)pending.size() < cfg.max_batch && age * 1e6 < cfg.window_us) break;
            const bool counts = pending.front().r.op == FS_REQ_COUNT;
            mode = counts ? FS_BATCH_COUNT : FS_BATCH_LENGTHS;
            for (auto it = pending.begin(); it != pending.end() && (int)take.size() < cfg.max_batch;) {
                if ((it->r.op == FS_REQ_COUNT) == counts) {
                    take.push_back(*it);
                    it = pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        std::vector<fs_query> qs(take.size());
        for (size_t i = 0; i < take.size(); i++) {
            qs[i].n = take[i].r.n;
            qs[i].d = take[i].r.d;
            memcpy(qs[i].gens, take[i].r.gens, sizeof qs[i].gens);
        }
        fs_status s = fs_batch_load_mode(sl.b, qs.data(), (int)qs.size(), mode, sl.st);
        int k = (int)qs.size();
        while (s == FS_E_CAPACITY && k > 1) {  // tables too large together: fewer queries
            k = (k + 1) / 2;
            s = fs_batch_load_mode(sl.b, qs.data(), k, mode, sl.st);
        }
        if (k < (int)take.size()) {
            // back to the queue, ahead of everything that came after them
            std::lock_guard<std::mutex> lk(mu);
            auto pos = pending.begin();
            while (pos != pending.end() && pos->ticket < take[k].ticket) ++pos;
            pending.insert(pos, take.begin() + k, take.end());
            take.resize(k);
        }
        if (s != FS_OK) {
            for (const Req& q : take) finish(q, s, 0, 0, 0, nullptr);
            progress = true;
            continue;
        }
        const double ts = now();
        for (Req& q : take) q.t_start = ts;
        s = fs_batch_launch(sl.b, sl.st);
        if (s == FS_OK) s = fs_batch_fetch(sl.b, sl.st);
        if (s != FS_OK) {
            for (const Req& q : take) finish(q, s, 0, 0, 0, nullptr);
            progress = true;
            continue;
        }
        cudaEventRecord(sl.ev, sl.st);
        sl.reqs = std::move(take);
        sl.busy = true;
        progress = true;
    }
    return progress;
}

void fs_server::run()
{
    cudaSetDevice(dev);
    for (;;) {
        const bool progress = step();
        std::unique_lock<std::mutex> lk(mu);
        const bool inflight = !job_wait.empty() || busy_gpu();
        if (stop && pending.empty() && !inflight) break;
        if (!progress) {
            if (pending.empty() && !inflight)
                cv_in.wait_for(lk, std::chrono::milliseconds(5));
            else
                cv_in.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

extern "C" {

fs_status fs_server_create(const fs_server_config* cfg, fs_server** out)
{
    if (!out) return FS_E_INVAL;
    fs_server* s = new fs_server;
    memset(&s->cfg, 0, sizeof s->cfg);
    if (cfg) s->cfg = *cfg;
    if (s->cfg.mem_budget_bytes == 0) s->cfg.mem_budget_bytes = 1ull << 30;
    if (s->cfg.max_batch <= 0) s->cfg.max_batch = 512;
    if (s->cfg.slots <= 0) s->cfg.slots = 3;
    if (s->cfg.window_us <= 0) s->cfg.window_us = 200;
    if (s->cfg.job_streams <= 0) s->cfg.job_streams = 4;
    if (s->cfg.hist_max_leaves == 0) s->cfg.hist_max_leaves = 1ull << 34;
    if (s->cfg.direct_leaves == 0) s->cfg.direct_leaves = 1ull << 24;
    if (s->cfg.table_bytes == 0) s->cfg.table_bytes = 256ull << 20;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&s->dev);
    fs_status st = e == cudaSuccess ? FS_OK : FS_E_CUDA;
    for (int i = 0; st == FS_OK && i < s->cfg.slots; i++) {
        Slot sl;
        st = fs_batch_reserve(s->cfg.max_batch, s->cfg.table_bytes, FS_BATCH_LENGTHS, nullptr, &sl.b);
        if (st != FS_OK) break;
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess)
            st = FS_E_CUDA;
        s->slots.push_back(sl);
    }
    if (st == FS_OK && fsi::dev_alloc((void**)&s->pool.base, s->cfg.mem_budget_bytes) != cudaSuccess)
        st = FS_E_NOMEM;
    for (int i = 0; st == FS_OK && i < s->cfg.job_streams; i++) {
        JobLane l;
        if (fsi::dev_alloc((void**)&l.dscratch, 3 * 8) != cudaSuccess ||
            fsi::host_alloc((void**)&l.hres, 3 * 8) != cudaSuccess)
            st = FS_E_NOMEM;
        else if (cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess ||
                 cudaEventCreateWithFlags(&l.ev, cudaEventDisableTiming) != cudaSuccess)
            st = FS_E_CUDA;
        s->lanes.push_back(l);
        if (st == FS_OK) st = fs_reserve(64ull << 20, l.st);  // each job stream's scratch
    }
    s->pool.size = s->cfg.mem_budget_bytes;
    s->pool.free_blocks[0] = s->cfg.mem_budget_bytes;
    if (st != FS_OK) {
        cudaGetLastError();
        s->stop = true;
        fs_server_destroy(s);
        return st;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return FS_OK;
}

fs_status fs_server_submit(fs_server* s, const fs_request* r, uint64_t* ticket)
{
    if (!s || !r || !ticket) return FS_E_INVAL;
    if (r->op < FS_REQ_COUNT || r->op > FS_REQ_ENUMERATE) return FS_E_INVAL;
    if (r->op == FS_REQ_ENUMERATE && r->elem_bytes != 2 && r->elem_bytes != 4) return FS_E_INVAL;
    if (r->op == FS_REQ_LENGTHS && r->hist != 0 && r->hist != 1) return FS_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return FS_E_INVAL;
    Req q;
    q.ticket = s->next_ticket++;
    q.r = *r;
    q.t_submit = s->now();
    q.t_start = q.t_counted = q.t_job = 0;
    q.direct = r->op != FS_REQ_ENUMERATE && batch_walk_leaves(*r) > (double)s->cfg.direct_leaves;
    s->pending.push_back(q);
    *ticket = q.ticket;
    s->cv_in.notify_one();
    return FS_OK;
}

fs_status fs_server_poll(fs_server* s, fs_response* out, int max, int* got, int wait_ms)
{
    if (!s || !out || !got || max < 1) return FS_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [s] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *got = k;
    return FS_OK;
}

fs_status fs_server_release(fs_server* s, uint64_t ticket)
{
    if (!s) return FS_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->held.find(ticket);
    if (it == s->held.end()) return FS_E_INVAL;
    s->pool.release(it->second.first, it->second.second);
    s->held.erase(it);
    s->cv_in.notify_one();
    return FS_OK;
}

fs_status fs_server_destroy(fs_server* s)
{
    if (!s) return FS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // rows still held by the caller are freed with the pool
        s->held.clear();
        s->pool.free_blocks.clear();
        s->pool.free_blocks[0] = s->pool.size;
        s->cv_in.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    for (Slot& sl : s->slots) {
        if (sl.b) fs_batch_destroy(sl.b);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
    }
    if (s->pool.base) cudaFree(s->pool.base);
    for (JobLane& l : s->lanes) {
        if (l.dscratch) cudaFree(l.dscratch);
        if (l.hres) cudaFreeHost(l.hres);
        if (l.st) cudaStreamDestroy(l.st);
        if (l.ev) cudaEventDestroy(l.ev);
    }
    delete s;
    return FS_OK;
}

}  // extern "C"
