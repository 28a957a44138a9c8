// Batched queries: thousands of (n, g) of uneven size in one persistent walk
// launch.  Every query is cut into slices of at most `target` leaves (target
// chosen from the total so that the batch has about items_target work items),
// so all work items are of comparable size and the device queue balances them
// regardless of how the work is distributed over queries.
//
//  k_batch_tables  one block per query: pair tables and leaf counts W, L_q
//  k_batch_plan    one block: target, slices per query, item offsets (scan)
//  k_batch_starts  one warp per item: the item's query, slice and start state
//  k_batch_walk    persistent warps: walk items, count (+ min / max length)
#include "launch.h"
#include "walk.cuh"

namespace fsi {

// The query a work item walks: q, or for trailing-k queries q with k - 2
// prefix levels fewer (the last k levels then come from the tables).  Copied
// word by word by the `nt` threads t = 0..nt-1 that call it (a warp or a
// block; one thread alone would load the whole structure in sequence), then
// reduced by thread 0; the caller synchronises those threads after it.
FS_D void batch_walk_query_copy(const BatchQ& B, QueryConst& out, int t, int nt)
{
    const uint32_t* src = (const uint32_t*)&B.q;
    uint32_t* dst = (uint32_t*)&out;
    for (int w = t; w < (int)(sizeof(QueryConst) / 4); w += nt) dst[w] = src[w];
}
FS_D void batch_walk_query_reduce(const BatchQ& B, QueryConst& out)
{
    if (B.trail) reduce_to_trailing(out, B.trail);
}

__global__ void __launch_bounds__(256) k_batch_tables(BatchDev b)
{
    __shared__ uint64_t part[256];
    __shared__ int32_t part32[256];
    __shared__ QueryConst qw;
    BatchQ& B = b.qs[blockIdx.x];
    if (!B.valid) return;
    batch_walk_query_copy(B, qw, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) batch_walk_query_reduce(B, qw);
    __syncthreads();
    if (B.trail) {
        trailing_tables_block(B.q, B.trail, (uint64_t*)(b.arena + B.off_T3),
                            b.mode ? (int32_t*)(b.arena + B.off_MN3) : nullptr,
                            b.mode ? (int32_t*)(b.arena + B.off_MX3) : nullptr, part, part32);
    } else {
        const QueryConst& q = B.q;
        int8_t* E = q.tab_e ? (int8_t*)(b.arena + B.off_E) : nullptr;
        int32_t* X0 = (b.mode && q.tab_xy) ? (int32_t*)(b.arena + B.off_X0) : nullptr;
        int32_t* YD = (b.mode && q.tab_xy) ? (int32_t*)(b.arena + B.off_YD) : nullptr;
        if (E || X0) pair_tables_fill(q, E, X0, YD, threadIdx.x, blockDim.x);
    }
    uint64_t* W = (uint64_t*)(b.arena + B.off_W);
    const int len = qw.n + 1;
    for (int k = qw.P - 2; k >= 0; k--) {
        const uint64_t* in = (k == qw.P - 2) ? nullptr : W + (size_t)(k + 1) * len;
        block_strided_prefix_sum(in, qw.dv_in, W + (size_t)k * len, len, qw.h[k], part);
    }
    __syncthreads();
    if (threadIdx.x == 0) B.L = total_leaves(qw, W);
}

// target = max(min_leaves, ceil(sum L / items_target)); S_q = ceil(L_q / target);
// item0 = exclusive scan of S_q; ctr[BCTR_ITEMS] = sum S_q.  One block.
__global__ void __launch_bounds__(1024) k_batch_plan(BatchDev b)
{
    __shared__ uint64_t part[1024];
    const int T = blockDim.x, tid = threadIdx.x;
    const int per = (b.nq + T - 1) / T;
    const int i0 = tid * per, i1 = min(b.nq, i0 + per);
    uint64_t sl = 0;
    for (int i = i0; i < i1; i++)
        if (b.qs[i].valid) sl += b.qs[i].L;
    part[tid] = sl;
    __syncthreads();
    for (int o = T / 2; o > 0; o >>= 1) {
        if (tid < o) part[tid] += part[tid + o];
        __syncthreads();
    }
    const uint64_t total = part[0];
    __syncthreads();
    uint64_t target = (total + b.items_target - 1) / b.items_target;
    if (target < b.min_leaves) target = b.min_leaves;
    uint64_t ss = 0;
    for (int i = i0; i < i1; i++) {
        BatchQ& B = b.qs[i];
        B.S = B.valid ? (B.L + target - 1) / target : 0;
        ss += B.S;
    }
    part[tid] = ss;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        const uint64_t v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint64_t run = tid > 0 ? part[tid - 1] : 0;
    for (int i = i0; i < i1; i++) {
        b.qs[i].item0 = run;
        run += b.qs[i].S;
    }
    if (tid == T - 1) {
        uint64_t items = part[T - 1];
        if (items > b.items_cap) {  // cannot happen: sum S_q <= items_target + nq
            atomicOr((unsigned long long*)&b.ctr[BCTR_ERR], 2ull);
            items = b.items_cap;
        }
        b.ctr[BCTR_ITEMS] = items;
    }
}

// The query of item `it`: the last q with item0[q] <= it (queries without
// items share their successor's item0 and are never the last such q).  A
// 32-way search by the calling warp (item0 never decreases; item0[0] = 0):
// each round the lanes probe 32 evenly spaced queries at once.
FS_D int batch_query_of(const BatchDev& b, uint64_t it, int lane)
{
    int lo = 0, hi = b.nq;  // answer in [lo, hi), item0[lo] <= it
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int probe = lo + lane * step;
        const bool ok = probe < hi && b.qs[probe].item0 <= it;
        const unsigned m = __ballot_sync(FULL, ok);  // lane 0 always
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_batch_starts(BatchDev b)
{
    __shared__ QueryConst qs[8];
    const int lane = threadIdx.x & 31;
    QueryConst& qw = qs[threadIdx.x >> 5];
    const uint64_t items = b.ctr[BCTR_ITEMS];
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    int cur = -1;
    for (uint64_t it = gw; it < items; it += nw) {
        const int j = batch_query_of(b, it, lane);
        const BatchQ& B = b.qs[j];
        if (j != cur) {
            __syncwarp();
            batch_walk_query_copy(B, qw, lane, 32);
            __syncwarp();
            if (lane == 0) batch_walk_query_reduce(B, qw);
            __syncwarp();
            cur = j;
        }
        const uint64_t s = it - B.item0;
        const uint64_t k0 = slice_start(s, B.L, B.S);
        RunPrefix rp;
        const int32_t bb = warp_unrank(qw, qw.h, qw.dv_h, (const uint64_t*)(b.arena + B.off_W),
                                       k0, lane, rp);
        int32_t* st = b.starts + it * START_W;
        if (lane < qw.P - 1) st[lane] = rp.a;
        if (lane == 0) {
            st[START_W - 3] = (int32_t)s;
            st[START_W - 2] = j;
            st[START_W - 1] = bb;
        }
    }
}

// count (+ min / max length) of one query, accumulated per lane
template <int MODE>
struct BatchCons {
    const int8_t* E;
    const int32_t* X0;
    const int32_t* YD;
    const uint64_t* T3;   // TRIPLE query: the trailing-three tables
    const int32_t* MN3;
    const int32_t* MX3;
    int triple;
    PairC pc;
    int tab;  // table path usable for this query and mode
    uint64_t cnt;
    uint32_t mn, mx;
    uint64_t* ctr;
    static constexpr int UNROLL = 2;
    // common-divisor skipping: a leaf's residual must be a multiple of the gcd
    // of the generators after the walk's innermost level (the last pair, or
    // the trailing three / four for a trailing-table query)
    static constexpr bool SKIP = true;
    static constexpr bool ANY_ORDER = true;
    static constexpr bool MULTI_SET = true;
    static constexpr uint32_t CHUNK_OPS = MODE ? 24 : 12;
    static constexpr bool R_INDEXED = false;
    FS_D void fault()
    {
        if ((threadIdx.x & 31) == 0) atomicOr((unsigned long long*)&ctr[BCTR_ERR], 1ull);
    }
    FS_D void group_begin(const QueryConst&, const RunPrefix&, int, int32_t, int32_t) {}
    FS_D bool chunk(const QueryConst&, int, bool valid, int32_t r, int32_t a, int32_t lp)
    {
        if (!valid) return false;
        if (triple) {
            const uint64_t c = __ldg(&T3[r]);
            cnt += c;
            if (MODE && c) {
                mn = min(mn, (uint32_t)(lp + a + __ldg(&MN3[r])));
                mx = max(mx, (uint32_t)(lp + a + __ldg(&MX3[r])));
            }
            return false;
        }
        if (MODE == 0) {
            cnt += tab ? pair_count<true>(pc, E, r) : pair_count<false>(pc, E, r);
        } else {
            int32_t x0 = 0, y0 = 0;
            const uint32_t c = tab ? pair_xy<true>(pc, X0, YD, r, x0, y0)
                                   : pair_xy<false>(pc, X0, YD, r, x0, y0);
            if (c > 0) {
                cnt += c;
                const int32_t l0 = lp + a + x0 + y0;
                const int32_t lt = l0 + (int32_t)(c - 1) * pc.delta;
                mn = min(mn, (uint32_t)min(l0, lt));
                mx = max(mx, (uint32_t)max(l0, lt));
            }
        }
        return false;
    }
};

// Count mode: four 256-thread blocks per SM (64 registers), since the walk
// waits on its per-query table loads and more resident warps hide more of
// that latency; the length mode keeps its registers (it spills at 64).
template <int MODE>
__global__ void __launch_bounds__(256, MODE ? 3 : 4) k_batch_walk(BatchDev b)
{
    __shared__ QueryConst qw[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    QueryConst& q = qw[wid];
    const uint64_t items = b.ctr[BCTR_ITEMS];
    const uint64_t W = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long* qc = (unsigned long long*)&b.ctr[BCTR_QUEUE];
    int cur = -1;
    int32_t hk = 0;
    BatchCons<MODE> cons;
    cons.ctr = b.ctr;
    uint64_t it = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    while (it < items) {
        unsigned long long nxt = 0;
        if (lane == 0) nxt = atomicAdd(qc, 1ull) + W;
        const int32_t* st = b.starts + it * START_W;
        const int j = st[START_W - 2];
        const uint64_t s = (uint64_t)st[START_W - 3];
        const BatchQ& B = b.qs[j];
        if (j != cur) {
            __syncwarp();
            const uint32_t* src = (const uint32_t*)&B.q;
            uint32_t* dst = (uint32_t*)&q;
            for (int w = lane; w < (int)(sizeof(QueryConst) / 4); w += 32) dst[w] = src[w];
            __syncwarp();
            cur = j;
            cons.pc = pair_consts(q);
            cons.tab = MODE == 0 ? q.tab_e : q.tab_xy;
            cons.triple = B.trail != 0;
            __syncwarp();
            if (B.trail && lane == 0) reduce_to_trailing(q, B.trail);
            __syncwarp();
            hk = lane < q.P - 1 ? q.h[lane] : 0;
            cons.E = (const int8_t*)(b.arena + B.off_E);
            cons.X0 = (const int32_t*)(b.arena + B.off_X0);
            cons.YD = (const int32_t*)(b.arena + B.off_YD);
            cons.T3 = (const uint64_t*)(b.arena + B.off_T3);
            cons.MN3 = (const int32_t*)(b.arena + B.off_MN3);
            cons.MX3 = (const int32_t*)(b.arena + B.off_MX3);
        }
        cons.cnt = 0;
        cons.mn = 0xffffffffu;
        cons.mx = 0;
        const uint64_t L = B.L, S = B.S;
        const uint64_t k0 = slice_start(s, L, S), k1 = slice_start(s + 1, L, S);
        if (k1 > k0) walk_slice(q, q.h, q.dv_h, b.starts, it, k1 - k0, lane, hk, cons);
        uint64_t c = warp_sum_u64(cons.cnt);
        uint32_t mn = cons.mn, mx = cons.mx;
        if (MODE) {
            for (int o = 16; o > 0; o >>= 1) {
                mn = min(mn, __shfl_xor_sync(FULL, mn, o));
                mx = max(mx, __shfl_xor_sync(FULL, mx, o));
            }
        }
        if (lane == 0 && c > 0) {
            BatchRes* R = &b.res[j];
            atomicAdd(&R->count, (unsigned long long)c);
            if (MODE) {
                atomicMax(&R->minc, (unsigned long long)(0xffffffffu - mn));
                atomicMax(&R->max, (unsigned long long)mx);
            }
        }
        it = __shfl_sync(FULL, nxt, 0);
    }
}

cudaError_t batch_walk_occupancy(int mode, int threads, int* nb)
{
    return occupancy_cached(mode ? (const void*)k_batch_walk<1> : (const void*)k_batch_walk<0>,
                            threads, 0, nb);
}

cudaError_t launch_batch(const BatchDev& b, int threads, int blocks, cudaStream_t st)
{
    k_batch_tables<<<b.nq, 256, 0, st>>>(b);
    k_batch_plan<<<1, 1024, 0, st>>>(b);
    uint64_t sb = (b.items_cap + 7) / 8;
    if (sb > 4096) sb = 4096;
    k_batch_starts<<<(unsigned)sb, 256, 0, st>>>(b);
    if (b.mode) k_batch_walk<1><<<blocks, threads, 0, st>>>(b);
    else k_batch_walk<0><<<blocks, threads, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace fsi
