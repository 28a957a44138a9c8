// Serving: a request loop with continuous batching, built on the batch-slot
// and enumerate entry points of the C ABI.
//
// Requests (count, length range, enumerate) are queued by fs_server_submit.
// One worker thread admits them into reusable batch slots, each with its own
// stream: a slot takes whatever has arrived (up to max_batch queries) as soon
// as it is free, so requests that arrive while other batches are on the GPU
// are batched and run concurrently with them.  Per-query planning state and
// slice queues stay on the device inside the slot.  An enumerate request is
// counted in a batch first; its rows are admitted only when count * d * bytes
// fits the server's device memory budget (else it is refused with
// FS_E_CAPACITY), then materialised into the budget's pool on an enumerate
// stream.  Completed requests are collected by fs_server_poll with
// submit / start / done timestamps.
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
    double t_start;
};

struct Slot {
    fs_batch* b = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Req> reqs;
    std::vector<fs_result> res;
};

struct EnumJob {
    Req req;
    uint64_t count;
    uint32_t min_len, max_len;
    uint64_t off, bytes;
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
    Pool pool;
    std::deque<EnumJob> enum_wait;
    bool enum_busy = false;
    EnumJob enum_cur;
    cudaStream_t enum_st = nullptr;
    cudaEvent_t enum_ev = nullptr;
    uint64_t* enum_dcount = nullptr;
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
        r.t_done = now();
        std::lock_guard<std::mutex> lk(mu);
        done.push_back(r);
        cv_done.notify_all();
    }

    bool step();
    void run();
};

bool fs_server::step()
{
    bool progress = false;
    // 1. finished batches
    for (Slot& sl : slots) {
        if (!sl.busy || cudaEventQuery(sl.ev) != cudaSuccess) continue;
        sl.res.resize(sl.reqs.size());
        fs_status s = fs_batch_collect(sl.b, sl.res.data());
        for (size_t i = 0; i < sl.reqs.size(); i++) {
            const Req& q = sl.reqs[i];
            const fs_result& R = sl.res[i];
            const int32_t st = s != FS_OK ? s : R.status;
            if (q.r.op == FS_REQ_ENUMERATE && st == FS_OK) {
                EnumJob j;
                j.req = q;
                j.count = R.count;
                j.min_len = R.min_len;
                j.max_len = R.max_len;
                j.off = 0;
                j.bytes = R.count * (uint64_t)q.r.d * (uint64_t)q.r.elem_bytes;
                enum_wait.push_back(j);
            } else {
                finish(q, st, R.count, R.min_len, R.max_len, nullptr);
            }
        }
        sl.reqs.clear();
        sl.busy = false;
        progress = true;
    }
    // 2. finished enumerate
    if (enum_busy && cudaEventQuery(enum_ev) == cudaSuccess) {
        {
            std::lock_guard<std::mutex> lk(mu);
            held[enum_cur.req.ticket] = {enum_cur.off, enum_cur.bytes};
        }
        finish(enum_cur.req, FS_OK, enum_cur.count, enum_cur.min_len, enum_cur.max_len,
               pool.base + enum_cur.off);
        enum_busy = false;
        progress = true;
    }
    // 3. start an enumerate: admitted by its exact output size
    while (!enum_busy && !enum_wait.empty()) {
        EnumJob& j = enum_wait.front();
        if (j.bytes > pool.size) {
            finish(j.req, FS_E_CAPACITY, j.count, j.min_len, j.max_len, nullptr);
            enum_wait.pop_front();
            progress = true;
            continue;
        }
        bool ok;
        {
            std::lock_guard<std::mutex> lk(mu);
            ok = pool.alloc(j.bytes, &j.off);
        }
        if (!ok) break;  // wait for rows to be released
        j.req.t_start = now();
        fs_config ec;
        fs_config_default(&ec);
        ec.keep_order = j.req.r.keep_order;
        fs_status s = fs_enumerate_async(j.req.r.n, j.req.r.gens, j.req.r.d, &ec,
                                         pool.base + j.off, j.count, j.req.r.elem_bytes,
                                         enum_dcount, enum_st);
        if (s != FS_OK) {
            std::lock_guard<std::mutex> lk(mu);
            pool.release(j.off, j.bytes);
        }
        if (s != FS_OK) {
            finish(j.req, s, j.count, j.min_len, j.max_len, nullptr);
            enum_wait.pop_front();
            continue;
        }
        cudaEventRecord(enum_ev, enum_st);
        enum_cur = j;
        enum_busy = true;
        enum_wait.pop_front();
        progress = true;
    }
    // 4. admit arrived requests into a free slot
    for (Slot& sl : slots) {
        if (sl.busy) continue;
        std::vector<Req> take;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (pending.empty()) break;
            // while other batches are on the GPU, let the batch fill for up to
            // window_us; an idle GPU takes what has arrived at once
            bool gpu_busy = enum_busy;
            for (const Slot& o : slots) gpu_busy = gpu_busy || o.busy;
            const double age = now() - pending.front().t_submit;
            if (gpu_busy && (int)pending.size() < cfg.max_batch && age * 1e6 < cfg.window_us) break;
            const int k = std::min<int>((int)pending.size(), cfg.max_batch);
            take.assign(pending.begin(), pending.begin() + k);
            pending.erase(pending.begin(), pending.begin() + k);
        }
        std::vector<fs_query> qs(take.size());
        for (size_t i = 0; i < take.size(); i++) {
            qs[i].n = take[i].r.n;
            qs[i].d = take[i].r.d;
            memcpy(qs[i].gens, take[i].r.gens, sizeof qs[i].gens);
        }
        fs_status s = fs_batch_load(sl.b, qs.data(), (int)qs.size(), sl.st);
        int k = (int)qs.size();
        while (s == FS_E_CAPACITY && k > 1) {  // tables too large together: fewer queries
            k = (k + 1) / 2;
            s = fs_batch_load(sl.b, qs.data(), k, sl.st);
        }
        if (k < (int)take.size()) {
            std::lock_guard<std::mutex> lk(mu);
            pending.insert(pending.begin(), take.begin() + k, take.end());
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
        bool inflight = enum_busy || !enum_wait.empty();
        for (const Slot& sl : slots) inflight = inflight || sl.busy;
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
    if (st == FS_OK) {
        if (fsi::dev_alloc((void**)&s->pool.base, s->cfg.mem_budget_bytes) != cudaSuccess ||
            fsi::dev_alloc((void**)&s->enum_dcount, 8) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s->enum_st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->enum_ev, cudaEventDisableTiming) != cudaSuccess)
            st = FS_E_NOMEM;
        if (st == FS_OK) st = fs_reserve(64ull << 20, s->enum_st);  // the enumerates' scratch
        s->pool.size = s->cfg.mem_budget_bytes;
        s->pool.free_blocks[0] = s->cfg.mem_budget_bytes;
    }
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
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return FS_E_INVAL;
    Req q;
    q.ticket = s->next_ticket++;
    q.r = *r;
    q.t_submit = s->now();
    q.t_start = 0;
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
    if (s->enum_dcount) cudaFree(s->enum_dcount);
    if (s->enum_st) cudaStreamDestroy(s->enum_st);
    if (s->enum_ev) cudaEventDestroy(s->enum_ev);
    delete s;
    return FS_OK;
}

}  // extern "C"
