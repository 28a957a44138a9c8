// The C ABI (include/fs.h): argument checks, canonical walk order, per-query
// constants, the device scratch arena, and the launch sequence of each
// consumer.  Every step of the computation runs in the kernels; this file
// only validates, lays out memory and enqueues.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"
#include "walk.cuh"

using namespace fsi;

namespace {

thread_local std::string t_err;

fs_status fail(fs_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

fs_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(FS_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// per-device state: scratch arena and a pinned result buffer
// ---------------------------------------------------------------------------
// Scratch of the calls on one stream of a device.
struct Arena {
    void* p = nullptr;
    size_t size = 0;
};

struct DevState {
    std::map<cudaStream_t, Arena> arenas;  // one scratch arena per stream
    uint64_t* pinned = nullptr;
    int sms = 0;
    // fs_enumerate_host: two device staging buffers, a copy stream, events
    void* stage = nullptr;
    size_t stage_size = 0;
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_comp[2] = {nullptr, nullptr};
    cudaEvent_t ev_copy[2] = {nullptr, nullptr};
};

std::mutex g_mu;
std::vector<DevState> g_dev;

fs_status get_dev(DevState** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DevState& ds = g_dev[dev];
    if (ds.sms == 0) {
        e = cudaDeviceGetAttribute(&ds.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        e = host_alloc((void**)&ds.pinned, 4096);
        if (e != cudaSuccess) {
            ds.sms = 0;
            return fail(FS_E_NOMEM, "cudaMallocHost: %s", cudaGetErrorString(e));
        }
    }
    *out = &ds;
    return FS_OK;
}

// The scratch arena of `st` on this device, at least `bytes` long.  Calls on
// one stream are ordered by it, so they can share its arena; calls on
// different streams have separate arenas and may overlap on the GPU.
fs_status ensure_arena(DevState* ds, cudaStream_t st, size_t bytes, void** out)
{
    Arena& a = ds->arenas[st];
    if (a.size >= bytes) {
        *out = a.p;
        return FS_OK;
    }
    if (a.p) {
        cudaStreamSynchronize(st);  // earlier work on this stream may still use it
        cudaFree(a.p);
        a.p = nullptr;
        a.size = 0;
    }
    size_t want = std::max(bytes, (size_t)16 << 20);
    want = (want + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
    cudaError_t e = dev_alloc(&a.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        a.p = nullptr;
        return fail(FS_E_NOMEM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
    }
    a.size = want;
    *out = a.p;
    return FS_OK;
}

// ---------------------------------------------------------------------------
// kernel timing (fs_profile_enable / fs_profile_read)
// ---------------------------------------------------------------------------
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
    int kernels;
};
bool g_prof = false;
std::string g_prof_only;  // record only scopes of this name (empty: all)
std::vector<ProfRec> g_prof_pending;

struct ProfScope {
    ProfRec rec;
    cudaStream_t st;
    bool on;
    ProfScope(const char* name, cudaStream_t s, int kernels)
        : st(s), on(g_prof && kernels > 0 && (g_prof_only.empty() || g_prof_only == name))
    {
        if (!on) return;
        rec.name = name;
        rec.kernels = kernels;
        cudaEventCreate(&rec.a);
        cudaEventCreate(&rec.b);
        cudaEventRecord(rec.a, st);
    }
    ~ProfScope()
    {
        if (!on) return;
        cudaEventRecord(rec.b, st);
        g_prof_pending.push_back(rec);
    }
};

// ---------------------------------------------------------------------------
// query canonicalisation and constants
// ---------------------------------------------------------------------------
int64_t gcd64(int64_t a, int64_t b)
{
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// inverse of a modulo m (gcd(a, m) = 1, m >= 1) by the extended Euclidean algorithm
int64_t modinv(int64_t a, int64_t m)
{
    if (m == 1) return 0;
    int64_t r0 = m, r1 = ((a % m) + m) % m, s0 = 0, s1 = 1;
    while (r1) {
        int64_t qt = r0 / r1, t = r0 - qt * r1;
        r0 = r1;
        r1 = t;
        t = s0 - qt * s1;
        s0 = s1;
        s1 = t;
    }
    return ((s0 % m) + m) % m;
}

struct Query {
    QueryConst q;
    std::vector<int> real_levels;  // walk levels with a caller column, in walk order
};

fs_status build_query(int64_t n, const uint32_t* gens, int d, const fs_config& cfg, Query& Q)
{
    if (!gens) return fail(FS_E_INVAL, "gens is NULL");
    if (d < 1 || d > FS_MAX_D) return fail(FS_E_INVAL, "d = %d outside [1, %d]", d, FS_MAX_D);
    if (n < 0) return fail(FS_E_INVAL, "n = %lld is negative", (long long)n);
    uint32_t gmax = 0, gmin = 0xffffffffu;
    for (int i = 0; i < d; i++) {
        if (gens[i] == 0) return fail(FS_E_INVAL, "generator %d is zero", i);
        gmax = std::max(gmax, gens[i]);
        gmin = std::min(gmin, gens[i]);
    }
    if (n + (int64_t)gmax > 2147483647LL)
        return fail(FS_E_OVERFLOW, "n + max g = %lld exceeds 2^31 - 1", (long long)(n + gmax));
    // Counts and leaf counts are uint64.  Every factorization is fixed by its
    // first d-1 coordinates (in any order), and each such prefix x with
    // sum x_i g_i <= n owns the unit cube [x, x+1), which lies in the simplex
    // sum y_i g_i <= n + sum g_i; so |Z| and the leaf counts are at most
    //   (n + sum g_i)^(d-1) / ((d-1)! prod g_i)   (the d-1 largest generators).
    // Queries whose bound reaches 2^63 are refused rather than risk a wrap.
    if (d >= 2) {
        std::vector<uint32_t> gs(gens, gens + d);
        std::sort(gs.begin(), gs.end(), std::greater<uint32_t>());
        long double lg = 0.0L, sum = 0.0L;
        for (int i = 0; i < d - 1; i++) sum += gs[i];
        for (int i = 0; i < d - 1; i++)
            lg += logl(((long double)n + sum) / (long double)gs[i]) - logl((long double)(i + 1));
        if (lg >= 63.0L * logl(2.0L))
            return fail(FS_E_OVERFLOW,
                        "the factorization count may exceed 2^63 (bound 2^%.1f): not representable",
                        (double)(lg / logl(2.0L)));
    }
    if (cfg.walk < FS_WALK_AUTO || cfg.walk > FS_WALK_LANES)
        return fail(FS_E_INVAL, "walk = %d: not an fs_walk", cfg.walk);
    if (cfg.reserved != 0) return fail(FS_E_INVAL, "fs_config.reserved = %d: must be 0", cfg.reserved);
    QueryConst& q = Q.q;
    memset(&q, 0, sizeof q);
    q.n = (int32_t)n;
    q.walk = cfg.walk;
    q.d = d;
    q.D = std::max(d, 3);
    q.P = q.D - 2;
    // walk order: caller's order, or descending generators (fewest prefixes)
    std::vector<int> ord(d);
    for (int i = 0; i < d; i++) ord[i] = i;
    if (!cfg.keep_order)
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return gens[a] > gens[b]; });
    const int32_t virt = (int32_t)n + 1;  // a generator above n: its coordinate is always 0
    std::vector<int> lev_col(q.D, -1);
    if (d >= 3) {
        for (int k = 0; k < d; k++) lev_col[k] = ord[k];
    } else if (d == 2) {
        lev_col[1] = ord[0];
        lev_col[2] = ord[1];
    } else {
        lev_col[1] = ord[0];
    }
    for (int k = 0; k < FS_MAX_D; k++) {
        q.col[k] = -1;
        q.h[k] = 1;
    }
    Q.real_levels.clear();
    for (int k = 0; k < q.D; k++) {
        q.col[k] = lev_col[k];
        q.h[k] = lev_col[k] >= 0 ? (int32_t)gens[lev_col[k]] : virt;
        if (lev_col[k] >= 0) Q.real_levels.push_back(k);
    }
    for (int k = 0; k < FS_MAX_D; k++) q.dv_h[k] = make_div32((uint32_t)q.h[k]);
    // the pair
    q.A = q.h[q.P];
    q.B = q.h[q.P + 1];
    const int64_t G = gcd64(q.A, q.B);
    q.G = (int32_t)G;
    q.u = (int32_t)(q.A / G);
    q.v = (int32_t)(q.B / G);
    q.inv = (int32_t)modinv(q.u, q.v);
    q.delta = q.v - q.u;
    const uint64_t lcm = (uint64_t)q.u * (uint64_t)q.B;
    q.tab_e = lcm <= (uint64_t)TABLE_E_MAX;
    q.tab_xy = lcm <= (uint64_t)TABLE_XY_MAX;
    q.lcm = (q.tab_e || q.tab_xy) ? (uint32_t)lcm : 0;
    if (q.lcm) q.dv_lcm = make_div32(q.lcm);
    q.dv_in = make_div32((uint32_t)q.h[q.P - 1]);
    q.dv_A = make_div32((uint32_t)q.A);
    q.dv_B = make_div32((uint32_t)q.B);
    q.dv_G = make_div32((uint32_t)q.G);
    q.dv_v = make_div32((uint32_t)q.v);
    q.maxlen = (int32_t)(n / gmin);
    q.dbins = q.maxlen + std::abs(q.delta) + 1;
    q.nw = q.P - 1;
    q.acc32 = q.lcm && 32.0 * ((double)n / q.h[q.P - 1] + 1.0) * ((double)n / q.lcm + 1.0) <
                           4294967295.0;
    q.fdiv = q.lcm >= 2 && (uint64_t)n * q.lcm < (1ull << 32);
    q.lcm_m1 = q.fdiv ? (uint32_t)(((1ull << 32) + q.lcm - 1) / q.lcm) : 0u;
    // common-divisor skipping for the pair walk (trailing gcd G) and for the
    // trailing-three / trailing-four walks (gcd of the last three / four)
    {
        int64_t Gt = G;
        for (int k = 0; k < 3; k++) {
            const int inner = q.P - 1 - k;  // the walk's innermost level
            if (k > 0) Gt = gcd64(Gt, q.h[q.P - k]);
            int64_t g1 = 1, m = 1, inv = 0;
            if (inner >= 0) {
                g1 = gcd64(q.h[inner], Gt);
                m = Gt / g1;
                inv = m > 1 ? modinv((q.h[inner] / g1) % m, m) : 0;
            }
            q.sk_g[k] = (int32_t)g1;
            q.sk_m[k] = (int32_t)m;
            q.sk_inv[k] = (int32_t)inv;
            q.dv_skg[k] = make_div32((uint32_t)g1);
            q.dv_skm[k] = make_div32((uint32_t)m);
        }
    }
    // planner tables: nw * (n + 1) uint64
    const double wbytes = (double)q.nw * (double)(n + 1) * 8.0;
    if (wbytes > 8.0 * (1ull << 30))
        return fail(FS_E_OVERFLOW, "leaf-count tables would take %.1f GiB (limit 8 GiB)",
                    wbytes / (1ull << 30));
    return FS_OK;
}

fs_status build_pred(const Query& Q, const fs_predicate* p, PredConst& pc)
{
    const QueryConst& q = Q.q;
    if (!p) return fail(FS_E_INVAL, "predicate is NULL");
    if (p->modulus == 0 && (p->op < 0 || p->op > 2))
        return fail(FS_E_INVAL, "predicate op %d outside {0,1,2}", p->op);
    if (p->c > (1ll << 60) || p->c < -(1ll << 60)) return fail(FS_E_INVAL, "|c| > 2^60");
    if (p->modulus > 0x7fffffffu) return fail(FS_E_INVAL, "modulus >= 2^31");
    memset(&pc, 0, sizeof pc);
    for (int k = 0; k < q.D; k++) {
        int c = q.col[k];
        if (c >= 0) {
            int32_t w = p->w[c];
            if (w > (1 << 20) || w < -(1 << 20)) return fail(FS_E_INVAL, "|w[%d]| > 2^20", c);
            pc.w[k] = w;
        }
    }
    pc.c = p->c;
    pc.op = p->op;
    pc.modulus = (int32_t)p->modulus;
    pc.dw = pc.w[q.P] * (int64_t)q.v - pc.w[q.P + 1] * (int64_t)q.u;
    if (pc.modulus > 0) {
        const int64_t M = pc.modulus;
        const int64_t dm = ((pc.dw % M) + M) % M;
        pc.gM = dm == 0 ? M : gcd64(dm, M);
        pc.Mq = M / pc.gM;
        pc.invq = modinv(dm / pc.gM, pc.Mq);
    }
    return FS_OK;
}

fs_config cfg_or_default(const fs_config* cfg)
{
    fs_config c;
    memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    return c;
}

// The query the trailing-k walk runs over: the first D-k levels as prefix
// levels (k - 2 fewer than PAIR); the last k come from the trailing tables.
// Enumerate counts its slices run by run from the trailing-three table (n + 1
// uint64 entries) below this n, leaf by leaf above it.
constexpr int32_t RUNS_MAX_N = 1 << 20;
// ... and, while the leaf counts and the prefix-count tables fit in this much
// shared memory, builds them in each planner block and takes every slice's
// offset from them (one launch for tables, planner and offsets).
constexpr size_t PLAN_RUNS_SMEM_MAX = 200 * 1024;

// Trailing levels the tables can take for q under `method` (0: none).
// k = 3 needs D >= 4 (one prefix level left) and n < 2^27 (the length
// sentinels stay in int32); k = 4 needs D >= 5 and n < 2^22, so that a table
// entry, at most C(n + 3, 3) < 2^64, cannot overflow.  AUTO and QUAD take
// the deepest that applies; TRIPLE takes 3.
int trailing_levels(const QueryConst& q, int method)
{
    const bool k4 = q.D >= 5 && q.n < (1 << 22);
    const bool k3 = q.D >= 4 && q.n < (1 << 27);
    if (method == FS_METHOD_TRIPLE) return k3 ? 3 : 0;
    if (method == FS_METHOD_QUAD) return k4 ? 4 : 0;
    return k4 ? 4 : k3 ? 3 : 0;
}

QueryConst reduce_trailing(const QueryConst& q, int k)
{
    QueryConst r = q;
    reduce_to_trailing(r, k);
    return r;
}

// ---------------------------------------------------------------------------
// launch geometry and scratch layout
// ---------------------------------------------------------------------------
fs_status geometry(const QueryConst& q, const fs_config& cfg, Op op, int method, int eb, int sms,
                   LaunchCfg& lc)
{
    cudaError_t e;
    int bps = 0;
    if (method == FS_METHOD_PLAIN) {
        lc.threads = 128;
        e = plain_occupancy(q, op, lc.threads, &bps);
    } else if (method == FS_METHOD_TRIPLE) {
        const int tdef = triple_threads(q, op);
        int t = cfg.block_threads > 0 ? cfg.block_threads : tdef;
        if (t % 32 != 0 || t > tdef) return fail(FS_E_INVAL, "block_threads %d: need a multiple of 32, <= %d", t, tdef);
        lc.threads = t;
        e = triple_occupancy(q, op, lc.threads, &bps);
    } else {
        int t = cfg.block_threads > 0 ? cfg.block_threads : 256;
        if (t % 32 != 0 || t > 256) return fail(FS_E_INVAL, "block_threads %d: need a multiple of 32, <= 256", t);
        lc.threads = t;
        e = pair_occupancy(q, op, lc.threads, eb, &bps);
    }
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (bps < 1) return fail(FS_E_CUDA, "kernel does not fit on an SM");
    if (cfg.blocks_per_sm > 0) bps = std::min(bps, cfg.blocks_per_sm);
    lc.blocks = sms * bps;
    // Slice count: explicit, or (auto) as many as leave about MIN_LEAVES leaves
    // per slice, at most 32 (enumerate 8) slices per warp / 2 per thread
    // (PLAIN); the planner picks the final number on the device, where the leaf
    // count is.  Several slices per warp: the cost of a leaf varies with its
    // run's length and, for the enumerate walk, with its row count.
    uint64_t S;
    if (cfg.slices > 0) {
        S = (uint64_t)cfg.slices;
        lc.auto_s = 0;
    } else {
        // The PAIR walks of the order-free consumers take 32 slices per warp:
        // the slices' leaves are equal but their cost is not, and the last
        // ones decide when the walk ends (the heavy count query: 1.12 s at 8
        // per warp, 1.01 s at 32).  Enumerate keeps 8 (each slice ends with a
        // partial flush of its rows; fewer measured slower, more too), and so
        // do the trailing-table walks, whose few leaves would make slices of a
        // few thousand leaves (twice the time on one config-3 seed at 32).
        const uint64_t per_warp = (op == OP_ENUM || method == FS_METHOD_TRIPLE) ? 8 : 32;
        S = method == FS_METHOD_PLAIN ? (uint64_t)lc.blocks * lc.threads * 2
                                      : (uint64_t)lc.blocks * (lc.threads / 32) * per_warp;
        // The warp walks end their queue with a tail of short slices
        // (make_split): the warps that take the last slices decide when the
        // walk ends (single large query, write walk: 0.303 -> 0.292 ms; heavy
        // count query: QUAD walk 0.350 -> 0.325 ms, PAIR 0.99 -> 0.97 s).
        lc.auto_s = method == FS_METHOD_PLAIN ? 1 : 2;
    }
    lc.min_leaves = method == FS_METHOD_PLAIN ? 16 : 256;
    if (S > (1ull << 31)) return fail(FS_E_INVAL, "slices = %llu exceeds 2^31", (unsigned long long)S);
    lc.S = S;
    return FS_OK;
}

struct Layout {
    size_t ctr, W, E, X0, YD, cnt, off, blk, D, starts, T3, MN3, MX3, extra, total;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

Layout make_layout(const QueryConst& q, uint64_t S, size_t extra_bytes, bool triple = false)
{
    Layout L;
    size_t p = 0;
    L.ctr = p;
    p = al(p + CTR_N * 8);
    L.W = p;
    p = al(p + (size_t)q.nw * (size_t)(q.n + 1) * 8);
    L.E = p;
    p = al(p + (q.tab_e ? q.lcm : 0));
    L.X0 = p;
    p = al(p + (q.tab_xy ? (size_t)q.lcm * 4 : 0));
    L.YD = p;
    p = al(p + (q.tab_xy ? (size_t)q.lcm * 4 : 0));
    L.cnt = p;
    p = al(p + (size_t)S * 8);
    L.off = p;
    p = al(p + (size_t)(S + 1) * 8);
    L.blk = p;
    p = al(p + (size_t)(S / SLICE_GROUP + 2) * 8);
    L.D = p;
    p = al(p + (size_t)std::max(q.dbins, q.maxlen + 1) * 8);
    L.starts = p;
    p = al(p + (size_t)S * START_W * 4);
    const size_t tn = triple ? (size_t)q.n + 1 : 0;
    L.T3 = p;
    p = al(p + tn * 8);
    L.MN3 = p;
    p = al(p + tn * 4);
    L.MX3 = p;
    p = al(p + tn * 4);
    L.extra = p;
    p = al(p + extra_bytes);
    L.total = p;
    return L;
}

Scratch scratch_at(void* base, const Layout& L)
{
    char* b = (char*)base;
    Scratch s;
    s.ctr = (uint64_t*)(b + L.ctr);
    s.W = (uint64_t*)(b + L.W);
    s.E = (int8_t*)(b + L.E);
    s.X0 = (int32_t*)(b + L.X0);
    s.YD = (int32_t*)(b + L.YD);
    s.slice_cnt = (uint64_t*)(b + L.cnt);
    s.slice_off = (uint64_t*)(b + L.off);
    s.blk = nullptr;
    s.s_lo = 0;
    s.s_hi = ~0ull;
    s.row_lo = 0;
    s.D = (uint64_t*)(b + L.D);
    s.starts = (int32_t*)(b + L.starts);
    return s;
}

const char* walk_name(Op op, int method)
{
    static const char* pair[] = {"pair_count", "pair_slice_count", "pair_len", "pair_any", "pair_enum"};
    static const char* plain[] = {"plain_count", "plain_slice_count", "plain_len", "plain_any",
                                  "plain_enum"};
    static const char* triple[] = {"triple_count", "triple_slice_count", "triple_len", "", ""};
    static const char* quad[] = {"quad_count", "quad_slice_count", "quad_len", "", ""};
    return method == FS_METHOD_PLAIN    ? plain[op]
           : method == FS_METHOD_TRIPLE ? triple[op]
           : method == FS_METHOD_QUAD   ? quad[op]
                                        : pair[op];
}

cudaError_t launch_walk(const QueryConst& q, const Scratch& sc, Op op, int method, const LaunchCfg& lc,
                        int queue, const PredConst* pred, void* out, uint64_t cap, int eb,
                        cudaStream_t st)
{
    ProfScope ps(walk_name(op, method), st, 1);
    if (method == FS_METHOD_PLAIN) return launch_plain(q, sc, op, lc, queue, pred, out, cap, eb, st);
    return launch_pair(q, sc, op, lc, queue, pred, out, cap, eb, st);
}

// Everything a call enqueues: precompute, walk(s), finalisation.
struct Call {
    Query Q;
    QueryConst q3;  // trailing tables: the reduced query the walk runs over
    fs_config cfg;
    int method = FS_METHOD_PAIR;  // PLAIN, PAIR, or TRIPLE for the trailing-k tables
    int trail = 0;                // TRIPLE: k = 3 or 4 trailing levels in the tables
    bool runs = false;            // PAIR enumerate: per-slice counts run by run from T3
    bool fused = false;           // tables, planner and offsets (prefix counts) in one launch
    Op op = OP_COUNT;
    DevState* ds = nullptr;
    Scratch sc;
    Layout L;
    LaunchCfg lc;
    cudaStream_t st = nullptr;
    uint64_t* T3 = nullptr;
    int32_t* MN3 = nullptr;
    int32_t* MX3 = nullptr;
    const QueryConst& wq() const { return method == FS_METHOD_TRIPLE ? q3 : Q.q; }
};

// Host half of a call: query, method, launch geometry and scratch layout.
// lengths_only: an OP_LEN call that wants no histogram (TRIPLE can serve it)
fs_status prepare_host(Call& c, int64_t n, const uint32_t* gens, int d, const fs_config* cfg, Op op,
                       int eb, void* stream, size_t extra_bytes = 0, bool lengths_only = false)
{
    c.cfg = cfg_or_default(cfg);
    c.st = (cudaStream_t)stream;
    fs_status s = build_query(n, gens, d, c.cfg, c.Q);
    if (s != FS_OK) return s;
    if (c.cfg.method < FS_METHOD_AUTO || c.cfg.method > FS_METHOD_QUAD)
        return fail(FS_E_INVAL, "method %d", c.cfg.method);
    const bool op_ok = op == OP_COUNT || op == OP_SLICES || (op == OP_LEN && lengths_only);
    const int kmax = trailing_levels(c.Q.q, FS_METHOD_AUTO);
    if (c.cfg.method == FS_METHOD_PLAIN) {
        c.method = FS_METHOD_PLAIN;
    } else if (c.cfg.method == FS_METHOD_TRIPLE || c.cfg.method == FS_METHOD_QUAD) {
        c.trail = trailing_levels(c.Q.q, c.cfg.method);
        if (!op_ok || c.trail == 0)
            return fail(FS_E_NOTIMPL, "%s serves count / slice counts / min-max lengths with "
                                      "d >= %d and n < 2^%d only",
                        c.cfg.method == FS_METHOD_TRIPLE ? "TRIPLE" : "QUAD",
                        c.cfg.method == FS_METHOD_TRIPLE ? 4 : 5,
                        c.cfg.method == FS_METHOD_TRIPLE ? 27 : 22);
        c.method = FS_METHOD_TRIPLE;
    } else if (c.cfg.method == FS_METHOD_AUTO && op_ok && kmax > 0) {
        c.trail = kmax;
        c.method = FS_METHOD_TRIPLE;
    } else {
        c.method = FS_METHOD_PAIR;
    }
    const bool triple = c.method == FS_METHOD_TRIPLE;
    if (triple) c.q3 = reduce_trailing(c.Q.q, c.trail);
    // enumerate's first walk (per-slice counts) goes run by run over the
    // trailing-three table when the table is small
    c.runs = op == OP_ENUM && c.method == FS_METHOD_PAIR && c.Q.q.n < RUNS_MAX_N;
    c.fused = c.runs && plan_runs_smem_bytes(c.Q.q) <= PLAN_RUNS_SMEM_MAX;
    const QueryConst& qw = c.wq();
    s = get_dev(&c.ds);
    if (s != FS_OK) return s;
    // the enumerate count walk and write walk share the slicing: take the
    // geometry of the write walk for both
    s = geometry(qw, c.cfg, op == OP_ENUM && c.method == FS_METHOD_PAIR ? OP_ENUM : op, c.method,
                 eb, c.ds->sms, c.lc);
    if (s != FS_OK) return s;
    c.L = make_layout(qw, c.lc.S, extra_bytes, triple || c.runs);
    c.op = op;
    return FS_OK;
}

// Device half: the scratch at `base` (c.L.total bytes), counter reset,
// precompute and planner launches.
fs_status prepare_device(Call& c, void* base)
{
    const bool triple = c.method == FS_METHOD_TRIPLE;
    const QueryConst& qw = c.wq();
    const Op op = c.op;
    c.sc = scratch_at(base, c.L);
    if (c.runs && !c.fused) c.sc.blk = (uint64_t*)((char*)base + c.L.blk);
    if (triple || c.runs) {
        char* b = (char*)base;
        c.T3 = (uint64_t*)(b + c.L.T3);
        c.MN3 = (int32_t*)(b + c.L.MN3);
        c.MX3 = (int32_t*)(b + c.L.MX3);
    }
    cudaError_t e = cudaMemsetAsync(c.sc.ctr, 0, CTR_N * 8, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (c.fused) return FS_OK;  // tables and planner run inside enum_count_slices
    {
        ProfScope ps("precompute", c.st,
                     (qw.tab_e || qw.tab_xy || qw.nw > 0 || triple || c.runs) ? 1 : 0);
        const bool lens = op == OP_LEN;  // the length tables only where they are read
        if (triple)
            e = launch_precompute(qw, c.sc, c.st, &c.Q.q, c.trail, c.T3, lens ? c.MN3 : nullptr,
                                  lens ? c.MX3 : nullptr);
        else if (c.runs)
            e = launch_precompute(qw, c.sc, c.st, &c.Q.q, 3, c.T3, nullptr, nullptr);
        else
            e = launch_precompute(qw, c.sc, c.st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "precompute launch");
    {
        ProfScope ps("plan", c.st, 1);
        e = launch_plan(qw, c.sc, c.lc.S, c.lc.auto_s, c.lc.min_leaves, c.st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "planner launch");
    return FS_OK;
}

// Both halves, with the scratch in the device's shared arena.
fs_status prepare(Call& c, int64_t n, const uint32_t* gens, int d, const fs_config* cfg, Op op,
                  int eb, void* stream, size_t extra_bytes = 0, bool lengths_only = false)
{
    fs_status s = prepare_host(c, n, gens, d, cfg, op, eb, stream, extra_bytes, lengths_only);
    if (s != FS_OK) return s;
    void* arena = nullptr;
    s = ensure_arena(c.ds, c.st, c.L.total, &arena);
    if (s != FS_OK) return s;
    return prepare_device(c, arena);
}

fs_status read_ctr(Call& c)
{
    cudaError_t e = cudaMemcpyAsync(c.ds->pinned, c.sc.ctr, CTR_N * 8, cudaMemcpyDeviceToHost, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return cuda_fail(e, "kernel execution");
    if (c.ds->pinned[CTR_ERR] != 0)
        return fail(FS_E_CUDA, "internal error: a slice walk ran past the last leaf (flags %llx)",
                    (unsigned long long)c.ds->pinned[CTR_ERR]);
    return FS_OK;
}

cudaError_t call_walk(Call& c, Op op, int queue, const PredConst* pred, void* out, uint64_t cap,
                      int eb)
{
    if (c.method == FS_METHOD_TRIPLE) {
        ProfScope ps(walk_name(op, c.trail == 4 ? FS_METHOD_QUAD : FS_METHOD_TRIPLE), c.st,
                     triple_walk_kernels(c.q3, op));
        return launch_triple(c.q3, c.sc, op, c.lc, queue, c.T3, c.MN3, c.MX3,
                             op == OP_COUNT ? (uint64_t*)out : nullptr, c.st);
    }
    return launch_walk(c.Q.q, c.sc, op, c.method, c.lc, queue, pred, out, cap, eb, c.st);
}

fs_status do_count(Call& c, uint64_t* dev_count)
{
    // PAIR and trailing-table count walks copy the total to dev_count themselves
    const bool walk_publishes = c.method != FS_METHOD_PLAIN;
    cudaError_t e = call_walk(c, OP_COUNT, CTR_QUEUE, nullptr, walk_publishes ? dev_count : nullptr, 0, 4);
    if (e != cudaSuccess) return cuda_fail(e, "count launch");
    if (dev_count && !walk_publishes) {
        ProfScope ps("copy_result", c.st, 1);
        e = launch_copy_u64(c.sc.ctr + CTR_COUNT, dev_count, c.st);
        if (e != cudaSuccess) return cuda_fail(e, "copy launch");
    }
    return FS_OK;
}

// Enumerate, first walk and scan: every slice's count, then its row offset.
fs_status enum_count_slices(Call& c, uint64_t* dev_count)
{
    cudaError_t e;
    if (c.fused) {
        ProfScope ps("plan_runs", c.st, 1);
        e = launch_plan_runs(c.Q.q, c.sc, c.lc.S, c.lc.auto_s, c.lc.min_leaves, dev_count, c.st);
        if (e != cudaSuccess) return cuda_fail(e, "enumerate plan launch");
        return FS_OK;
    }
    if (c.runs) {
        // counts, offsets within groups of slices, and (last block) the
        // groups' offsets, in one launch
        ProfScope ps("pair_slice_runs", c.st, 1);
        e = launch_pair_slice_runs(c.Q.q, c.sc, c.T3, c.lc.S, dev_count, c.st);
        if (e != cudaSuccess) return cuda_fail(e, "enumerate count launch");
        return FS_OK;
    }
    e = launch_walk(c.Q.q, c.sc, OP_SLICES, c.method, c.lc, CTR_QUEUE, nullptr, nullptr, 0, 4, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "enumerate count launch");
    {
        ProfScope ps("scan_slices", c.st, 1);
        e = launch_scan_slices(c.sc, dev_count, c.st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "scan launch");
    return FS_OK;
}

// Enumerate, second walk: the rows of the slices in sc's window into dev_buf
// (cap rows from global row sc.row_lo on).
fs_status enum_write(Call& c, const Scratch& sc, void* dev_buf, uint64_t cap, int eb, cudaStream_t st)
{
    if (cap == 0) return FS_OK;
    cudaError_t e = launch_walk(c.Q.q, sc, OP_ENUM, c.method, c.lc, CTR_QUEUE2, nullptr, dev_buf, cap, eb, st);
    if (e != cudaSuccess) return cuda_fail(e, "enumerate write launch");
    return FS_OK;
}

fs_status do_enum(Call& c, void* dev_buf, uint64_t cap, int eb, uint64_t* dev_count)
{
    fs_status s = enum_count_slices(c, dev_count);
    if (s == FS_OK) s = enum_write(c, c.sc, dev_buf, cap, eb, c.st);
    return s;
}

// The slices [s0, s1) that hold rows [pos, pos + rows) of the ordered
// output, from the host copy of the slice offsets (off[0..S]).
void window_slices(const std::vector<uint64_t>& off, uint64_t S, uint64_t pos, uint64_t rows,
                   uint64_t* s0, uint64_t* s1)
{
    const auto b = off.begin(), e = off.begin() + (ptrdiff_t)S + 1;
    *s0 = (uint64_t)(std::upper_bound(b, e, pos) - b) - 1;
    *s1 = (uint64_t)(std::lower_bound(b, e, pos + rows) - b);
}

// Rows [pos, pos + rows) of the ordered output into dev_buf: the write walk
// over the slices that hold them, rows outside the window dropped.
fs_status enum_window(Call& c, const std::vector<uint64_t>& off, uint64_t S, uint64_t pos,
                      uint64_t rows, void* dev_buf, int eb, cudaStream_t st)
{
    Scratch sc = c.sc;
    window_slices(off, S, pos, rows, &sc.s_lo, &sc.s_hi);
    sc.row_lo = pos;
    cudaError_t e = cudaMemsetAsync(&c.sc.ctr[CTR_QUEUE2], 0, 8, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    return enum_write(c, sc, dev_buf, rows, eb, st);
}

// The slice offsets to the host after enum_count_slices (synchronises c.st).
fs_status fetch_offsets(Call& c, uint64_t* S, uint64_t* total, std::vector<uint64_t>& off)
{
    fs_status s = read_ctr(c);
    if (s != FS_OK) return s;
    *S = c.ds->pinned[CTR_SEFF];
    *total = c.ds->pinned[CTR_TOTAL];
    off.resize(*S + 1);
    std::vector<uint64_t> blk(c.sc.blk ? *S / SLICE_GROUP + 1 : 0);
    cudaError_t e = cudaMemcpyAsync(off.data(), c.sc.slice_off, *S * 8, cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess && c.sc.blk)
        e = cudaMemcpyAsync(blk.data(), c.sc.blk, blk.size() * 8, cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return cuda_fail(e, "slice offsets to host");
    if (c.sc.blk)
        for (uint64_t s = 0; s < *S; s++) off[s] += blk[s / SLICE_GROUP];
    off[*S] = *total;
    return FS_OK;
}

fs_status check_enum_args(const Query& Q, void* dev_buf, uint64_t cap, int eb)
{
    if (eb != 2 && eb != 4) return fail(FS_E_INVAL, "elem_bytes = %d, need 2 or 4", eb);
    if (cap > 0 && !dev_buf) return fail(FS_E_INVAL, "dev_buf is NULL");
    if (((uintptr_t)dev_buf & 15) != 0) return fail(FS_E_INVAL, "dev_buf is not 16-byte aligned");
    if (eb == 2 && Q.q.maxlen > 32767)
        return fail(FS_E_OVERFLOW, "int16 output: a coordinate can reach %d", Q.q.maxlen);
    if (cap > (~0ull) / (uint64_t)Q.q.d / 4) return fail(FS_E_INVAL, "cap too large");
    return FS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void fs_config_default(fs_config* cfg)
{
    if (cfg) memset(cfg, 0, sizeof *cfg);
}

const char* fs_status_string(int s)
{
    switch (s) {
    case FS_OK: return "FS_OK";
    case FS_E_INVAL: return "FS_E_INVAL";
    case FS_E_OVERFLOW: return "FS_E_OVERFLOW";
    case FS_E_CAPACITY: return "FS_E_CAPACITY";
    case FS_E_NOMEM: return "FS_E_NOMEM";
    case FS_E_CUDA: return "FS_E_CUDA";
    case FS_E_TIMEOUT: return "FS_E_TIMEOUT";
    case FS_E_NOTIMPL: return "FS_E_NOTIMPL";
    }
    return "FS_E_UNKNOWN";
}

int fs_version(void) { return 100; }

const char* fs_last_error(void) { return t_err.c_str(); }

fs_status fs_count_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                      uint64_t* out_count, void* stream)
{
    if (!out_count) return fail(FS_E_INVAL, "out_count is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    Call c;
    fs_status s = prepare(c, n, gens, d, cfg, OP_COUNT, 4, stream);
    if (s == FS_OK) s = do_count(c, nullptr);
    if (s == FS_OK) s = read_ctr(c);
    if (s == FS_OK) *out_count = c.ds->pinned[CTR_COUNT];
    return s;
}

fs_status fs_count(int64_t n, const uint32_t* gens, int d, uint64_t* out_count, void* stream)
{
    return fs_count_ex(n, gens, d, nullptr, out_count, stream);
}

fs_status fs_count_async(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                         uint64_t* dev_count, void* stream)
{
    if (!dev_count) return fail(FS_E_INVAL, "dev_count is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    Call c;
    fs_status s = prepare(c, n, gens, d, cfg, OP_COUNT, 4, stream);
    if (s == FS_OK) s = do_count(c, dev_count);
    return s;
}

// Enqueues the length walk of a prepared call: the TRIPLE / QUAD walk for the
// count and length range alone, else the PAIR (or PLAIN) walk into the
// difference array and its finalisation, which takes the count and range from
// the histogram.  Either way the counters hold count, min and max afterwards.
static fs_status enqueue_lengths(Call& c, uint64_t* hist_dev)
{
    const QueryConst& q = c.Q.q;
    cudaError_t e;
    if (c.method == FS_METHOD_TRIPLE) {
        e = call_walk(c, OP_LEN, CTR_QUEUE, nullptr, nullptr, 0, 4);
        if (e != cudaSuccess) return cuda_fail(e, "length launch");
        return FS_OK;
    }
    e = cudaMemsetAsync(c.sc.D, 0, (size_t)std::max(q.dbins, q.maxlen + 1) * 8, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = call_walk(c, OP_LEN, CTR_QUEUE, nullptr, nullptr, 0, 4);
    if (e != cudaSuccess) return cuda_fail(e, "length launch");
    const int stride = c.method == FS_METHOD_PLAIN ? 0 : std::abs(q.delta);
    ProfScope ps("len_finalize", c.st, 1);
    e = launch_len_finalize(q, c.sc, hist_dev, stride, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "finalize launch");
    return FS_OK;
}

fs_status fs_length_stats_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                             fs_len_summary* out, uint64_t* hist_dev, void* stream)
{
    if (!out) return fail(FS_E_INVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    Call c;
    fs_status s = prepare(c, n, gens, d, cfg, OP_LEN, 4, stream, 0, hist_dev == nullptr);
    if (s != FS_OK) return s;
    s = enqueue_lengths(c, hist_dev);
    if (s != FS_OK) return s;
    s = read_ctr(c);
    if (s != FS_OK) return s;
    out->count = c.ds->pinned[CTR_COUNT];
    if (out->count > 0) {
        out->min_len = (uint32_t)(0xffffffffu - c.ds->pinned[CTR_MINC]);
        out->max_len = (uint32_t)c.ds->pinned[CTR_MAX];
    } else {
        out->min_len = out->max_len = 0;
    }
    return FS_OK;
}

fs_status fs_length_stats_async(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                                uint64_t* hist_dev, uint64_t* out_dev, void* stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    Call c;
    fs_status s = prepare(c, n, gens, d, cfg, OP_LEN, 4, stream, 0, hist_dev == nullptr);
    if (s != FS_OK) return s;
    s = enqueue_lengths(c, hist_dev);
    if (s != FS_OK) return s;
    if (out_dev) {
        const cudaError_t e = launch_len_summary(c.sc, out_dev, c.st);
        if (e != cudaSuccess) return cuda_fail(e, "summary launch");
    }
    return FS_OK;
}

fs_status fs_length_stats(int64_t n, const uint32_t* gens, int d, fs_len_summary* out,
                          uint64_t* hist_dev, void* stream)
{
    return fs_length_stats_ex(n, gens, d, nullptr, out, hist_dev, stream);
}

fs_status fs_any_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                    const fs_predicate* pred, int* out_bool, void* stream)
{
    if (!out_bool) return fail(FS_E_INVAL, "out_bool is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    Call c;
    fs_config cc = cfg_or_default(cfg);
    // validate the predicate before any device work
    {
        Query Q;
        fs_status s = build_query(n, gens, d, cc, Q);
        if (s != FS_OK) return s;
        PredConst pc;
        s = build_pred(Q, pred, pc);
        if (s != FS_OK) return s;
    }
    fs_status s = prepare(c, n, gens, d, cfg, OP_ANY, 4, stream);
    if (s != FS_OK) return s;
    PredConst pc;
    s = build_pred(c.Q, pred, pc);
    if (s != FS_OK) return s;
    cudaError_t e = launch_walk(c.Q.q, c.sc, OP_ANY, c.method, c.lc, CTR_QUEUE, &pc, nullptr, 0, 4, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "any launch");
    s = read_ctr(c);
    if (s == FS_OK) *out_bool = c.ds->pinned[CTR_FOUND] ? 1 : 0;
    return s;
}

fs_status fs_any(int64_t n, const uint32_t* gens, int d, const fs_predicate* pred, int* out_bool,
                 void* stream)
{
    return fs_any_ex(n, gens, d, nullptr, pred, out_bool, stream);
}

fs_status fs_enumerate_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                          void* dev_buf, uint64_t cap, int elem_bytes, uint64_t* out_count,
                          void* stream)
{
    if (!out_count) return fail(FS_E_INVAL, "out_count is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    {
        Query Q;
        fs_status s = build_query(n, gens, d, cfg_or_default(cfg), Q);
        if (s != FS_OK) return s;
        s = check_enum_args(Q, dev_buf, cap, elem_bytes);
        if (s != FS_OK) return s;
    }
    Call c;
    fs_status s = prepare(c, n, gens, d, cfg, OP_ENUM, elem_bytes, stream);
    if (s == FS_OK) s = do_enum(c, dev_buf, cap, elem_bytes, nullptr);
    if (s == FS_OK) s = read_ctr(c);
    if (s != FS_OK) return s;
    *out_count = c.ds->pinned[CTR_TOTAL];
    if (*out_count > cap)
        return fail(FS_E_CAPACITY, "%llu factorizations, capacity %llu",
                    (unsigned long long)*out_count, (unsigned long long)cap);
    return FS_OK;
}

fs_status fs_enumerate(int64_t n, const uint32_t* gens, int d, void* dev_buf, uint64_t cap,
                       int elem_bytes, uint64_t* out_count, void* stream)
{
    return fs_enumerate_ex(n, gens, d, nullptr, dev_buf, cap, elem_bytes, out_count, stream);
}

fs_status fs_enumerate_async(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                             void* dev_buf, uint64_t cap, int elem_bytes, uint64_t* dev_count,
                             void* stream)
{
    if (!dev_count) return fail(FS_E_INVAL, "dev_count is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    {
        Query Q;
        fs_status s = build_query(n, gens, d, cfg_or_default(cfg), Q);
        if (s != FS_OK) return s;
        s = check_enum_args(Q, dev_buf, cap, elem_bytes);
        if (s != FS_OK) return s;
    }
    Call c;
    fs_status s = prepare(c, n, gens, d, cfg, OP_ENUM, elem_bytes, stream);
    if (s == FS_OK) s = do_enum(c, dev_buf, cap, elem_bytes, dev_count);
    return s;
}

// ---------------------------------------------------------------------------
// resumable cursor and streamed enumerate
// ---------------------------------------------------------------------------
}  // extern "C"

struct fs_cursor {
    Call c;
    void* mem = nullptr;  // the cursor's own scratch (c.L.total bytes)
    int eb = 4;
    uint64_t S = 0, total = 0, pos = 0;
    std::vector<uint64_t> off;  // row offset of every slice, S + 1 entries
};

namespace {

fs_status stage_ready(DevState* ds, size_t bytes)
{
    if (!ds->copy_st) {
        cudaError_t e = cudaStreamCreateWithFlags(&ds->copy_st, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; i++) {
            e = cudaEventCreateWithFlags(&ds->ev_comp[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ds->ev_copy[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "copy stream");
    }
    if (ds->stage_size >= bytes) return FS_OK;
    if (ds->stage) {
        cudaDeviceSynchronize();
        cudaFree(ds->stage);
        ds->stage = nullptr;
        ds->stage_size = 0;
    }
    cudaError_t e = dev_alloc(&ds->stage, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ds->stage = nullptr;
        return fail(FS_E_NOMEM, "staging cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    ds->stage_size = bytes;
    return FS_OK;
}

// Staging chunk of fs_enumerate_host: large enough that each window's launch
// is small beside its copy, small enough to overlap the next window's walk.
constexpr size_t STAGE_CHUNK_BYTES = 128u << 20;

}  // namespace

extern "C" {

fs_status fs_cursor_create(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                           int elem_bytes, void* stream, fs_cursor** out)
{
    if (!out) return fail(FS_E_INVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    {
        Query Q;
        fs_status s = build_query(n, gens, d, cfg_or_default(cfg), Q);
        if (s != FS_OK) return s;
        s = check_enum_args(Q, nullptr, 0, elem_bytes);
        if (s != FS_OK) return s;
    }
    fs_cursor* k = new fs_cursor;
    Call& c = k->c;
    fs_status s = prepare_host(c, n, gens, d, cfg, OP_ENUM, elem_bytes, stream);
    if (s == FS_OK && c.method != FS_METHOD_PAIR)
        s = fail(FS_E_NOTIMPL, "a cursor walks the PAIR method (method %d asked)", c.cfg.method);
    if (s == FS_OK) {
        cudaError_t e = dev_alloc(&k->mem, c.L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            k->mem = nullptr;
            s = fail(FS_E_NOMEM, "cursor cudaMalloc(%zu): %s", c.L.total, cudaGetErrorString(e));
        }
    }
    if (s == FS_OK) s = prepare_device(c, k->mem);
    if (s == FS_OK) s = enum_count_slices(c, nullptr);
    if (s == FS_OK) s = fetch_offsets(c, &k->S, &k->total, k->off);
    if (s != FS_OK) {
        if (k->mem) {
            cudaDeviceSynchronize();
            cudaFree(k->mem);
        }
        delete k;
        return s;
    }
    k->eb = elem_bytes;
    *out = k;
    return FS_OK;
}

fs_status fs_cursor_count(const fs_cursor* k, uint64_t* total)
{
    if (!k || !total) return fail(FS_E_INVAL, "cursor / total is NULL");
    *total = k->total;
    return FS_OK;
}

fs_status fs_cursor_tell(const fs_cursor* k, uint64_t* row)
{
    if (!k || !row) return fail(FS_E_INVAL, "cursor / row is NULL");
    *row = k->pos;
    return FS_OK;
}

fs_status fs_cursor_slices(const fs_cursor* k, uint64_t* slices)
{
    if (!k || !slices) return fail(FS_E_INVAL, "cursor / slices is NULL");
    *slices = k->S;
    return FS_OK;
}

fs_status fs_cursor_seek(fs_cursor* k, uint64_t row)
{
    if (!k) return fail(FS_E_INVAL, "cursor is NULL");
    if (row > k->total)
        return fail(FS_E_INVAL, "seek to row %llu of %llu", (unsigned long long)row,
                    (unsigned long long)k->total);
    k->pos = row;
    return FS_OK;
}

fs_status fs_cursor_next(fs_cursor* k, void* dev_buf, uint64_t cap, uint64_t* rows, void* stream)
{
    if (!k || !rows) return fail(FS_E_INVAL, "cursor / rows is NULL");
    if (cap > 0 && !dev_buf) return fail(FS_E_INVAL, "dev_buf is NULL");
    if (((uintptr_t)dev_buf & 15) != 0) return fail(FS_E_INVAL, "dev_buf is not 16-byte aligned");
    std::lock_guard<std::mutex> lk(g_mu);
    const uint64_t left = k->total - k->pos;
    const uint64_t m = cap < left ? cap : left;
    *rows = m;
    if (m == 0) return FS_OK;
    fs_status s = enum_window(k->c, k->off, k->S, k->pos, m, dev_buf, k->eb, (cudaStream_t)stream);
    if (s == FS_OK) k->pos += m;
    return s;
}

fs_status fs_cursor_destroy(fs_cursor* k)
{
    if (!k) return FS_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaError_t e = cudaDeviceSynchronize();
    if (k->mem) cudaFree(k->mem);
    delete k;
    if (e != cudaSuccess) return cuda_fail(e, "cursor free");
    return FS_OK;
}

fs_status fs_enumerate_host(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                            void* host_buf, uint64_t cap, int elem_bytes, uint64_t* out_count,
                            void* stream)
{
    if (!out_count) return fail(FS_E_INVAL, "out_count is NULL");
    if (cap > 0 && !host_buf) return fail(FS_E_INVAL, "host_buf is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    {
        Query Q;
        fs_status s = build_query(n, gens, d, cfg_or_default(cfg), Q);
        if (s != FS_OK) return s;
        s = check_enum_args(Q, nullptr, 0, elem_bytes);
        if (s != FS_OK) return s;
        if (cap > (~0ull) / (uint64_t)Q.q.d / 4) return fail(FS_E_INVAL, "cap too large");
    }
    Call c;
    fs_status s = prepare(c, n, gens, d, cfg, OP_ENUM, elem_bytes, stream);
    if (s == FS_OK && c.method != FS_METHOD_PAIR)
        s = fail(FS_E_NOTIMPL, "fs_enumerate_host walks the PAIR method (method %d asked)", c.cfg.method);
    if (s == FS_OK) s = enum_count_slices(c, nullptr);
    uint64_t S = 0, total = 0;
    std::vector<uint64_t> off;
    if (s == FS_OK) s = fetch_offsets(c, &S, &total, off);
    if (s != FS_OK) return s;
    *out_count = total;
    const uint64_t want = cap < total ? cap : total;
    const size_t row_bytes = (size_t)c.Q.q.d * (size_t)elem_bytes;
    if (want > 0) {
        uint64_t chunk = STAGE_CHUNK_BYTES / row_bytes;
        if (chunk > want) chunk = want;
        if (chunk < 1) chunk = 1;
        const size_t half = al((size_t)chunk * row_bytes);
        DevState* ds = c.ds;
        s = stage_ready(ds, 2 * half);
        if (s != FS_OK) return s;
        cudaError_t e = cudaSuccess;
        uint64_t k = 0;
        for (uint64_t pos = 0; pos < want && s == FS_OK && e == cudaSuccess; k++) {
            const uint64_t rows = chunk < want - pos ? chunk : want - pos;
            void* buf = (char*)ds->stage + (k & 1) * half;
            if (k >= 2) e = cudaStreamWaitEvent(c.st, ds->ev_copy[k & 1], 0);  // buffer drained
            if (e == cudaSuccess) s = enum_window(c, off, S, pos, rows, buf, elem_bytes, c.st);
            if (s != FS_OK) break;
            e = cudaEventRecord(ds->ev_comp[k & 1], c.st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ds->copy_st, ds->ev_comp[k & 1], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((char*)host_buf + pos * row_bytes, buf, rows * row_bytes,
                                    cudaMemcpyDeviceToHost, ds->copy_st);
            if (e == cudaSuccess) e = cudaEventRecord(ds->ev_copy[k & 1], ds->copy_st);
            pos += rows;
        }
        const cudaError_t e2 = cudaStreamSynchronize(ds->copy_st);
        if (s != FS_OK) return s;
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return cuda_fail(e, "streamed enumerate");
        s = read_ctr(c);  // the write walks' fault flag
        if (s != FS_OK) return s;
    }
    if (total > cap)
        return fail(FS_E_CAPACITY, "%llu factorizations, capacity %llu", (unsigned long long)total,
                    (unsigned long long)cap);
    return FS_OK;
}

fs_status fs_plan(int64_t n, const uint32_t* gens, int d, const fs_config* cfg, int64_t slices,
                  int32_t* order, int32_t* bounds, uint64_t* leaves)
{
    if (slices < 1 || slices > (1ll << 31)) return fail(FS_E_INVAL, "slices = %lld", (long long)slices);
    std::lock_guard<std::mutex> lk(g_mu);
    fs_config cc = cfg_or_default(cfg);
    cc.slices = slices;
    Call c;
    fs_status s = prepare(c, n, gens, d, &cc, OP_SLICES, 4, nullptr);
    if (s != FS_OK) return s;
    const QueryConst& q = c.wq();
    std::vector<int32_t> hs((size_t)slices * START_W);
    cudaError_t e = cudaMemcpyAsync(hs.data(), c.sc.starts, hs.size() * 4, cudaMemcpyDeviceToHost, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    s = read_ctr(c);
    if (s != FS_OK) return s;
    if (leaves) *leaves = c.ds->pinned[CTR_L];
    const int nr = (int)c.Q.real_levels.size();
    if (order)
        for (int j = 0; j < nr; j++) order[j] = q.col[c.Q.real_levels[j]];
    if (bounds) {
        for (int64_t sl = 0; sl < slices; sl++) {
            const int32_t* st = &hs[(size_t)sl * START_W];
            const bool empty = st[START_W - 1] < 0;
            for (int j = 0; j < nr; j++) {
                const int k = c.Q.real_levels[j];
                int32_t v = 0;
                if (k < q.P - 1) v = st[k];
                else if (k == q.P - 1) v = st[START_W - 1];
                bounds[sl * d + j] = empty ? -1 : v;
            }
        }
        for (int j = 0; j < d; j++) bounds[slices * d + j] = -1;
    }
    return FS_OK;
}

fs_status fs_slice_counts(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                          int64_t slices, uint64_t* counts, void* stream)
{
    if (!counts) return fail(FS_E_INVAL, "counts is NULL");
    if (slices < 1 || slices > (1ll << 31)) return fail(FS_E_INVAL, "slices = %lld", (long long)slices);
    std::lock_guard<std::mutex> lk(g_mu);
    fs_config cc = cfg_or_default(cfg);
    cc.slices = slices;
    Call c;
    fs_status s = prepare(c, n, gens, d, &cc, OP_SLICES, 4, stream);
    if (s != FS_OK) return s;
    cudaError_t e = call_walk(c, OP_SLICES, CTR_QUEUE, nullptr, nullptr, 0, 4);
    if (e != cudaSuccess) return cuda_fail(e, "slice count launch");
    e = cudaMemcpyAsync(counts, c.sc.slice_cnt, (size_t)slices * 8, cudaMemcpyDeviceToHost, c.st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return cuda_fail(e, "slice count execution");
    return FS_OK;
}

fs_status fs_reserve(uint64_t bytes, void* stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DevState* ds = nullptr;
    fs_status s = get_dev(&ds);
    if (s != FS_OK) return s;
    void* arena = nullptr;
    return ensure_arena(ds, (cudaStream_t)stream, (size_t)bytes, &arena);
}

void fs_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof = on != 0;
}

void fs_profile_only(const char* name)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof_only = name ? name : "";
}

int fs_profile_read(char* names, uint64_t* launches, double* total_ms, int max)
{
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<std::string> order;
    std::map<std::string, std::pair<uint64_t, double>> acc;
    int rc = 0;
    for (ProfRec& r : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            rc = -1;
        if (!acc.count(r.name)) order.push_back(r.name);
        acc[r.name].first += (uint64_t)r.kernels;
        acc[r.name].second += ms;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_pending.clear();
    if (rc < 0) {
        cudaGetLastError();
        return -1;
    }
    int k = 0;
    for (const std::string& nm : order) {
        if (k >= max) break;
        if (names) {
            strncpy(names + 32 * k, nm.c_str(), 31);
            names[32 * k + 31] = 0;
        }
        if (launches) launches[k] = acc[nm].first;
        if (total_ms) total_ms[k] = acc[nm].second;
        k++;
    }
    return k;
}

fs_status fs_probe_int_rate(int kind, uint32_t iters, double* ops_per_s)
{
    if (kind < 0 || kind > 2 || !ops_per_s || iters == 0) return fail(FS_E_INVAL, "bad probe arguments");
    std::lock_guard<std::mutex> lk(g_mu);
    double ms = 0;
    cudaError_t e = int_probe(kind, iters, ops_per_s, &ms);
    if (e != cudaSuccess) return cuda_fail(e, "integer probe");
    return FS_OK;
}

// ---------------------------------------------------------------------------
// batched queries
// ---------------------------------------------------------------------------
}  // extern "C"

struct fs_batch {
    int dev = -1;
    int nq = 0;          // queries loaded
    int cap_q = 0;       // queries reserved
    uint64_t cap_arena = 0;
    int mode = 0;
    fs_config cfg;
    std::vector<int32_t> status;
    void* mem = nullptr;
    BatchQ* hq = nullptr;       // pinned: constants to upload
    BatchRes* hres = nullptr;   // pinned: fetched results
    uint64_t* hctr = nullptr;   // pinned: fetched counters
    BatchDev bd;
    int threads = 256;
    int blocks = 0;
    int sms = 0;
};

namespace {

fs_status batch_shape(fs_batch* b, int threads, int blocks_per_sm, uint64_t items)
{
    if (threads <= 0) threads = 256;
    if (threads % 32 != 0 || threads > 256) return fail(FS_E_INVAL, "block_threads %d: need a multiple of 32, <= 256", threads);
    int bps = 0;
    cudaError_t e = batch_walk_occupancy(b->mode, threads, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (bps < 1) return fail(FS_E_CUDA, "batch kernel does not fit on an SM");
    if (blocks_per_sm > 0) bps = std::min(bps, blocks_per_sm);
    b->threads = threads;
    b->blocks = b->sms * bps;
    const uint64_t warps = (uint64_t)b->blocks * (threads / 32);
    uint64_t target = items > 0 ? items : warps * 8;
    if (target + (uint64_t)b->cap_q > b->bd.items_cap) target = b->bd.items_cap - (uint64_t)b->cap_q;
    if (target < 1) target = 1;
    b->bd.items_target = target;
    return FS_OK;
}

// Host-side planning of queries into BatchQ records (in `out`), their table
// offsets and statuses; returns the table bytes they need.
uint64_t batch_plan_host(const fs_query* queries, int nq, int mode, const fs_config& cc, BatchQ* out,
                         int32_t* status)
{
    uint64_t arena = 0;
    auto take = [&](size_t bytes) {
        const uint64_t o = arena;
        arena += (bytes + 15) & ~(size_t)15;
        return o;
    };
    fs_config walk_cfg = cfg_or_default(nullptr);  // descending walk order
    walk_cfg.walk = cc.walk;                         // the caller's sibling-group mode
    for (int i = 0; i < nq; i++) {
        BatchQ& B = out[i];
        memset(&B, 0, sizeof B);
        const fs_query& Q = queries[i];
        Query qq;
        fs_status s = FS_E_INVAL;
        if (Q.d >= 1 && Q.d <= FS_MAX_D) s = build_query(Q.n, Q.gens, Q.d, walk_cfg, qq);
        status[i] = s;
        if (s != FS_OK) continue;
        B.q = qq.q;
        B.valid = 1;
        // the trailing tables unless PAIR is asked for
        B.trail = cc.method == FS_METHOD_PAIR ? 0 : trailing_levels(B.q, cc.method);
        const size_t n1 = (size_t)B.q.n + 1;
        if (B.trail) {
            B.off_W = take((size_t)(B.q.nw - (B.trail - 2)) * n1 * 8);
            B.off_T3 = take(n1 * 8);
            B.off_MN3 = take(mode == FS_BATCH_LENGTHS ? n1 * 4 : 0);
            B.off_MX3 = take(mode == FS_BATCH_LENGTHS ? n1 * 4 : 0);
        } else {
            B.off_W = take((size_t)B.q.nw * n1 * 8);
            B.off_E = take(B.q.tab_e ? B.q.lcm : 0);
            const bool xy = mode == FS_BATCH_LENGTHS && B.q.tab_xy;
            B.off_X0 = take(xy ? (size_t)B.q.lcm * 4 : 0);
            B.off_YD = take(xy ? (size_t)B.q.lcm * 4 : 0);
        }
    }
    return arena;
}

void batch_free(fs_batch* b)
{
    if (b->mem) cudaFree(b->mem);
    if (b->hq) cudaFreeHost(b->hq);
    if (b->hres) cudaFreeHost(b->hres);
    delete b;
}

}  // namespace

extern "C" {

fs_status fs_batch_table_bytes(const fs_query* queries, int nq, int mode, const fs_config* cfg,
                               uint64_t* bytes)
{
    if (!queries || !bytes || nq < 1) return fail(FS_E_INVAL, "batch: queries / bytes NULL or nq < 1");
    std::vector<BatchQ> tmp(nq);
    std::vector<int32_t> st(nq);
    *bytes = batch_plan_host(queries, nq, mode, cfg_or_default(cfg), tmp.data(), st.data());
    return FS_OK;
}

fs_status fs_batch_reserve(int max_queries, uint64_t table_bytes, int mode, const fs_config* cfg,
                           fs_batch** out)
{
    if (!out || max_queries < 1) return fail(FS_E_INVAL, "batch: out NULL or max_queries < 1");
    if (mode != FS_BATCH_COUNT && mode != FS_BATCH_LENGTHS) return fail(FS_E_INVAL, "batch mode %d", mode);
    std::lock_guard<std::mutex> lk(g_mu);
    fs_config cc = cfg_or_default(cfg);
    fs_batch* b = new fs_batch;
    b->cap_q = max_queries;
    b->cap_arena = table_bytes;
    b->mode = mode;
    b->cfg = cc;
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "no CUDA device");
    }
    // items: room for the largest shape the autotuner tries (32 per warp at
    // the maximum occupancy of 256-thread blocks) or the requested count
    int bps = 0;
    batch_walk_occupancy(mode, 256, &bps);
    const uint64_t max_items = std::max<uint64_t>((uint64_t)std::max(cc.slices, (int64_t)0),
                                                  (uint64_t)b->sms * std::max(bps, 1) * 8 * 32);
    b->bd.items_cap = max_items + (uint64_t)max_queries;
    const size_t off_qs = 0;
    const size_t off_res = al(off_qs + sizeof(BatchQ) * (size_t)max_queries);
    const size_t off_ctr = al(off_res + sizeof(BatchRes) * (size_t)max_queries);
    const size_t off_st = al(off_ctr + BCTR_N * 8);
    const size_t off_ar = al(off_st + (size_t)b->bd.items_cap * START_W * 4);
    const size_t total = al(off_ar + table_bytes);
    e = dev_alloc(&b->mem, total);
    if (e == cudaSuccess) e = host_alloc((void**)&b->hq, sizeof(BatchQ) * (size_t)max_queries);
    if (e == cudaSuccess)
        e = host_alloc((void**)&b->hres, sizeof(BatchRes) * (size_t)max_queries + BCTR_N * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return fail(FS_E_NOMEM, "batch reserve (%zu device bytes): %s", total, cudaGetErrorString(e));
    }
    b->hctr = (uint64_t*)(b->hres + max_queries);
    char* base = (char*)b->mem;
    b->bd.qs = (BatchQ*)(base + off_qs);
    b->bd.nq = 0;
    b->bd.mode = mode;
    b->bd.arena = (unsigned char*)(base + off_ar);
    b->bd.starts = (int32_t*)(base + off_st);
    b->bd.ctr = (uint64_t*)(base + off_ctr);
    b->bd.res = (BatchRes*)(base + off_res);
    b->bd.min_leaves = 64;
    fs_status s = batch_shape(b, cc.block_threads, cc.blocks_per_sm, (uint64_t)std::max(cc.slices, (int64_t)0));
    if (s != FS_OK) {
        batch_free(b);
        return s;
    }
    *out = b;
    return FS_OK;
}

fs_status fs_batch_load(fs_batch* b, const fs_query* queries, int nq, void* stream)
{
    if (!b || !queries || nq < 1) return fail(FS_E_INVAL, "batch: NULL or nq < 1");
    if (nq > b->cap_q) return fail(FS_E_CAPACITY, "batch: %d queries, room for %d", nq, b->cap_q);
    std::lock_guard<std::mutex> lk(g_mu);
    b->status.assign(nq, FS_OK);
    const uint64_t need = batch_plan_host(queries, nq, b->mode, b->cfg, b->hq, b->status.data());
    if (need > b->cap_arena)
        return fail(FS_E_CAPACITY, "batch: tables need %llu bytes, room for %llu",
                    (unsigned long long)need, (unsigned long long)b->cap_arena);
    cudaError_t e = cudaMemcpyAsync(b->bd.qs, b->hq, sizeof(BatchQ) * (size_t)nq,
                                    cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch upload");
    b->nq = nq;
    b->bd.nq = nq;
    return FS_OK;
}

fs_status fs_batch_load_mode(fs_batch* b, const fs_query* queries, int nq, int mode, void* stream)
{
    if (!b) return fail(FS_E_INVAL, "batch is NULL");
    if (mode != FS_BATCH_COUNT && mode != FS_BATCH_LENGTHS) return fail(FS_E_INVAL, "batch mode %d", mode);
    if (mode != b->mode) {
        std::lock_guard<std::mutex> lk(g_mu);
        const int old = b->mode;
        b->mode = mode;
        b->bd.mode = mode;
        fs_status s = batch_shape(b, b->cfg.block_threads, b->cfg.blocks_per_sm,
                                  (uint64_t)std::max(b->cfg.slices, (int64_t)0));
        if (s != FS_OK) {
            b->mode = b->bd.mode = old;
            return s;
        }
    }
    return fs_batch_load(b, queries, nq, stream);
}

fs_status fs_batch_fetch(fs_batch* b, void* stream)
{
    if (!b || b->nq < 1) return fail(FS_E_INVAL, "batch: NULL or nothing loaded");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(b->hres, b->bd.res, sizeof(BatchRes) * (size_t)b->nq,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->hctr, b->bd.ctr, BCTR_N * 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch fetch");
    return FS_OK;
}

fs_status fs_batch_collect(fs_batch* b, fs_result* results)
{
    if (!b || !results) return fail(FS_E_INVAL, "batch / results is NULL");
    if (b->hctr[BCTR_ERR]) return fail(FS_E_CUDA, "internal error in the batch walk (flags %llx)",
                                       (unsigned long long)b->hctr[BCTR_ERR]);
    for (int i = 0; i < b->nq; i++) {
        fs_result& R = results[i];
        R.count = b->hres[i].count;
        R.status = b->status[i];
        R.pad = 0;
        if (b->mode == FS_BATCH_LENGTHS && R.count > 0) {
            R.min_len = (uint32_t)(0xffffffffu - b->hres[i].minc);
            R.max_len = (uint32_t)b->hres[i].max;
        } else {
            R.min_len = R.max_len = 0;
        }
    }
    return FS_OK;
}

fs_status fs_batch_create(const fs_query* queries, int nq, int mode, const fs_config* cfg,
                          fs_batch** out)
{
    if (!queries || !out || nq < 1) return fail(FS_E_INVAL, "batch: queries / out NULL or nq < 1");
    uint64_t bytes = 0;
    fs_status s = fs_batch_table_bytes(queries, nq, mode, cfg, &bytes);
    if (s != FS_OK) return s;
    fs_batch* b = nullptr;
    s = fs_batch_reserve(nq, bytes, mode, cfg, &b);
    if (s != FS_OK) return s;
    s = fs_batch_load(b, queries, nq, nullptr);
    if (s == FS_OK) {
        cudaError_t e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) s = cuda_fail(e, "batch upload");
    }
    if (s != FS_OK) {
        batch_free(b);
        return s;
    }
    *out = b;
    return FS_OK;
}

fs_status fs_batch_launch(fs_batch* b, void* stream)
{
    if (!b || b->nq < 1) return fail(FS_E_INVAL, "batch is NULL or has no queries loaded");
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope ps("batch", st, 4);
    cudaError_t e = cudaMemsetAsync(b->bd.ctr, 0, BCTR_N * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->bd.res, 0, sizeof(BatchRes) * (size_t)b->nq, st);
    if (e == cudaSuccess) e = launch_batch(b->bd, b->threads, b->blocks, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return FS_OK;
}

fs_status fs_batch_results(fs_batch* b, fs_result* results, void* stream)
{
    if (!b || !results) return fail(FS_E_INVAL, "batch / results is NULL");
    fs_status s = fs_batch_fetch(b, stream);
    if (s != FS_OK) return s;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch execution");
    return fs_batch_collect(b, results);
}

fs_status fs_batch_destroy(fs_batch* b)
{
    if (!b) return FS_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaError_t e = cudaDeviceSynchronize();
    batch_free(b);
    if (e != cudaSuccess) return cuda_fail(e, "batch free");
    return FS_OK;
}

fs_status fs_batch_run(const fs_query* queries, int nq, int mode, const fs_config* cfg,
                       fs_result* results, void* stream)
{
    fs_batch* b = nullptr;
    fs_status s = fs_batch_create(queries, nq, mode, cfg, &b);
    if (s != FS_OK) return s;
    s = fs_batch_launch(b, stream);
    if (s == FS_OK) s = fs_batch_results(b, results, stream);
    fs_status s2 = fs_batch_destroy(b);
    return s != FS_OK ? s : s2;
}

fs_status fs_batch_autotune(const fs_query* queries, int nq, int mode, fs_config* best,
                            double* best_ms, void* stream)
{
    if (!best) return fail(FS_E_INVAL, "best is NULL");
    fs_batch* b = nullptr;
    fs_status s = fs_batch_create(queries, nq, mode, nullptr, &b);
    if (s != FS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads_c[] = {128, 256};
    const int per_warp_c[] = {2, 4, 8, 16, 32};
    double best_t = 1e30;
    fs_config bc;
    memset(&bc, 0, sizeof bc);
    for (int t : threads_c)
        for (int pw : per_warp_c) {
            {
                std::lock_guard<std::mutex> lk(g_mu);
                int bps = 0;
                batch_walk_occupancy(b->mode, t, &bps);
                const uint64_t items = (uint64_t)b->sms * std::max(bps, 1) * (t / 32) * pw;
                s = batch_shape(b, t, 0, items);
            }
            if (s != FS_OK) break;
            s = fs_batch_launch(b, st);  // warm-up
            if (s != FS_OK) break;
            float ms = 1e30f;  // best of three
            for (int rep = 0; rep < 3 && s == FS_OK; rep++) {
                cudaEventRecord(e0, st);
                s = fs_batch_launch(b, st);
                cudaEventRecord(e1, st);
                if (s != FS_OK) break;
                cudaError_t e = cudaEventSynchronize(e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (e != cudaSuccess) s = cuda_fail(e, "autotune timing");
                ms = std::min(ms, t);
            }
            if (s != FS_OK) break;
            if (ms < best_t) {
                best_t = ms;
                bc.block_threads = t;
                bc.slices = (int64_t)b->bd.items_target;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fs_status s2 = fs_batch_destroy(b);
    if (s != FS_OK) return s;
    *best = bc;
    if (best_ms) *best_ms = best_t;
    return s2;
}

fs_status fs_selftest_split(uint64_t leaves, uint64_t slices, int tail, uint64_t* starts)
{
    if (slices == 0 || !starts) return FS_E_INVAL;
    const SliceSplit sp = make_split(leaves, slices, tail ? 2 : 1);
    for (uint64_t s = 0; s <= slices; s++) starts[s] = sp.start(s);
    return FS_OK;
}

int64_t fs_selftest_division(uint32_t div, uint32_t x0, uint32_t count)
{
    if (div == 0 || div > 0x7fffffffu) return -1;
    if ((uint64_t)x0 + count > 0x80000000ull) return -1;
    const Div32 q = make_div32(div);
    int64_t bad = 0;
    for (uint64_t x = x0; x < (uint64_t)x0 + count; x++) {
        uint32_t qq = div32((uint32_t)x, q);
        uint32_t rr = (uint32_t)x - qq * div;
        if (qq != (uint32_t)x / div || rr != (uint32_t)x % div) bad++;
    }
    return bad;
}

}  // extern "C"

// ===========================================================================
// Allocation-free count (fs_count_noalloc)
// ===========================================================================
// Its scratch is the static device array below instead of the cudaMalloc'd
// arena: every device that loads the library holds FS_NOALLOC_SCRATCH_BYTES
// of it until the process exits.  All calls share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FS_NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress while that device is current.
constexpr int NOALLOC_MAX_DEVICES = 64;
// slices of the allocation-free count: their start states take 64 bytes each
constexpr uint64_t NOALLOC_SLICES = 4096;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES];
}  // namespace

extern "C" fs_status fs_count_noalloc(int64_t n, const uint32_t* gens, int d, uint64_t* dev_count,
                                      void* stream)
{
    if (!dev_count) return fail(FS_E_INVAL, "dev_count is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    fs_config cfg = cfg_or_default(nullptr);
    Query Q;
    fs_status s = build_query(n, gens, d, cfg, Q);
    if (s != FS_OK) return s;
    QueryConst q = Q.q;
    q.tab_xy = 0;  // the count walk reads only the E table
    // scratch layout inside the static array: counters | leaf counts W | E table |
    // slice start states (at most NOALLOC_SLICES slices)
    const size_t off_W = al(CTR_N * 8);
    const size_t off_E = off_W + al((size_t)q.nw * (size_t)(q.n + 1) * 8);
    const size_t off_st = off_E + al(q.tab_e ? q.lcm : 0);
    const size_t need = off_st + al((size_t)NOALLOC_SLICES * START_W * 4);
    if (need > (size_t)FS_NOALLOC_SCRATCH_BYTES)
        return fail(FS_E_OVERFLOW,
                    "fs_count_noalloc: this query needs %zu bytes of scratch; the static maximum "
                    "is %zu bytes (FS_NOALLOC_SCRATCH_BYTES); use fs_count",
                    need, (size_t)FS_NOALLOC_SCRATCH_BYTES);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(FS_E_CUDA, "device %d out of range", dev);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_addr[dev] = ptr;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    LaunchCfg lc;
    s = geometry(q, cfg, OP_COUNT, FS_METHOD_PAIR, 4, sms, lc);
    if (s != FS_OK) return s;
    if (lc.S > NOALLOC_SLICES) lc.S = NOALLOC_SLICES;
    char* base = (char*)g_noalloc_addr[dev];
    Scratch sc;
    memset(&sc, 0, sizeof sc);
    sc.s_hi = ~0ull;
    sc.ctr = (uint64_t*)base;
    sc.W = (uint64_t*)(base + off_W);
    sc.E = (int8_t*)(base + off_E);
    sc.starts = (int32_t*)(base + off_st);
    cudaStream_t st = (cudaStream_t)stream;
    // the counters (slice queue head, total) must start at zero on every call
    const char* what = "cudaMemsetAsync";
    e = cudaMemsetAsync(sc.ctr, 0, CTR_N * 8, st);
    if (e == cudaSuccess) {
        what = "precompute launch";
        e = launch_precompute(q, sc, st);
    }
    if (e == cudaSuccess) {
        what = "planner launch";
        e = launch_plan(q, sc, lc.S, lc.auto_s, lc.min_leaves, st);
    }
    if (e == cudaSuccess) {
        what = "count launch";
        e = launch_pair(q, sc, OP_COUNT, lc, CTR_QUEUE, nullptr, nullptr, 0, 4, st);
    }
    if (e == cudaSuccess) {
        what = "copy launch";
        e = launch_copy_u64(sc.ctr + CTR_COUNT, dev_count, st);
    }
    if (e != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;  // looked up again by the next call
        return cuda_fail(e, what);
    }
    return FS_OK;
}
