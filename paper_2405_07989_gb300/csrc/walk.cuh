// Device-side building blocks of the bounded lexicographic walk.
//
// The lex order on the leaves (prefixes (a_0..a_{P-1}) with phi <= n, walk
// order, a_0 most significant) is cut into S slices of consecutive leaf ranks
// (Sec. 4: a bound splits the lex-ordered output between workers; here the
// bounds are clean prefixes (leaf, 0, 0), so each worker's stream starts at a
// state that satisfies the hypothesis of Thm 3.2, cf. Remark 4.2).  A warp
// takes one slice at a time, finds the slice's first leaf from the exact leaf
// counts W (the planner), and then walks the slice's leaves 32 per step, a
// group of sibling runs at a time: in lex order for enumerate, full steps run
// by run and the runs' remainders packed for the order-free consumers.
#pragma once

#include <cuda_runtime.h>

#include "fs_internal.h"

namespace fsi {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Slices: slice s holds the leaf ranks [start(s), start(s + 1)).  The first Sh
// slices split the first Lh leaves evenly (Lh = Q Sh + R, 0 <= R < Sh: the
// first R of them one leaf more); the remaining slices, the tail, split the
// other leaves evenly the same way (Qt, Rt).  Without a tail Sh = S, Lh = L.
// The walks take slices in index order from a dynamic queue, so a tail of
// short slices lets the warps finish close together.
// ---------------------------------------------------------------------------
struct SliceSplit {
    uint64_t Q, R, Sh, Lh, Qt, Rt;
    SliceSplit() = default;
    FS_HD SliceSplit(uint64_t L, uint64_t S) : Q(L / S), R(L % S), Sh(S), Lh(L), Qt(0), Rt(0) {}
    // The last St of the S slices hold 1/shrink of a head slice's leaves each.
    FS_HD static SliceSplit tailed(uint64_t L, uint64_t S, uint64_t St, uint32_t shrink)
    {
        if (St == 0 || St >= S || shrink <= 1) return SliceSplit(L, S);
        const double den = (double)shrink * (double)(S - St) + (double)St;
        uint64_t Lt = (uint64_t)((double)L * (double)St / den);
        if (Lt > L) Lt = L;
        SliceSplit p(L - Lt, S - St);
        p.Qt = Lt / St;
        p.Rt = Lt % St;
        return p;
    }
    FS_HD uint64_t start(uint64_t s) const
    {
        if (s <= Sh) return s * Q + (s < R ? s : R);
        const uint64_t t = s - Sh;
        return Lh + t * Qt + (t < Rt ? t : Rt);
    }
};

// The planner's split, as it recorded it (no 64-bit division per thread).
FS_D SliceSplit planned_split(const uint64_t* ctr)
{
    SliceSplit p;
    p.Q = ctr[CTR_SQ];
    p.R = ctr[CTR_SR];
    p.Sh = ctr[CTR_SH];
    p.Lh = ctr[CTR_LH];
    p.Qt = ctr[CTR_TQ];
    p.Rt = ctr[CTR_TR];
    return p;
}

// The split of L leaves into S slices as the planner makes it (auto_s == 2:
// with a tail of a sixteenth of the slices, each a sixteenth the size).
FS_HD SliceSplit make_split(uint64_t L, uint64_t S, int auto_s)
{
    return auto_s == 2 ? SliceSplit::tailed(L, S, S / 16, 16) : SliceSplit(L, S);
}

// Records the split for the walks (planned_split).
FS_D void record_split(uint64_t* ctr, const SliceSplit& sp)
{
    ctr[CTR_SQ] = sp.Q;
    ctr[CTR_SR] = sp.R;
    ctr[CTR_SH] = sp.Sh;
    ctr[CTR_LH] = sp.Lh;
    ctr[CTR_TQ] = sp.Qt;
    ctr[CTR_TR] = sp.Rt;
}

FS_HD uint64_t slice_start(uint64_t s, uint64_t L, uint64_t S)
{
    return SliceSplit(L, S).start(s);
}

// Number of leaves: W_0[n], or for a single prefix level floor(n / h_0) + 1.
FS_D uint64_t total_leaves(const QueryConst& q, const uint64_t* W)
{
    if (q.P == 1) return (uint64_t)div32((uint32_t)q.n, q.dv_in) + 1;
    return W[q.n];
}

// ---------------------------------------------------------------------------
// Block-wide strided prefix sum: out[p] = sum_{j >= 0, p - j*s >= 0} in(p - j*s)
// for p in [0, len), i.e. out[p] = in(p) + out[p - s].  Multiplying a series by
// 1/(1 - x^s) -- the recurrence behind the leaf counts (W_k[p] = W_{k+1}[p] +
// W_k[p - h_k]) and behind the strided difference array of the length
// histogram.  `in` may be NULL, in which case in(p) = floor(p / s_in) + 1 (the
// closed-form count of the innermost prefix level).  Must be called by all
// threads of the block; uses T * 8 bytes of shared scratch `part`.
// ---------------------------------------------------------------------------
FS_D uint64_t sps_in(const uint64_t* in, int p, const Div32& dv_in)
{
    return in ? in[p] : (uint64_t)div32((uint32_t)p, dv_in) + 1;
}

// Few, short chains (a small table): one warp per chain, no block-wide
// barriers (which is what the segmented form below spends its time on at this
// size).  A chain of up to 256 elements is scanned in one pass: lane l takes
// the E = ceil(len_chain / 32) consecutive elements from l E on (their loads
// all in flight at once), sums them, and a warp scan of the lane totals
// places them.
FS_D bool strided_by_warps(int len, int s)
{
    return s <= 2 * (int)(blockDim.x >> 5) && (len - 1) / s + 1 <= 256;
}

template <class T, class Op, class In>
FS_D void warp_chains_scan(In in, T* out, int len, int s, Op op, T ident)
{
    constexpr int EMAX = 8;  // 256 / 32
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int rho = threadIdx.x >> 5; rho < s; rho += nw) {
        const int cl = (len - 1 - rho) / s + 1;  // elements rho, rho + s, .. below len
        const int E = (cl + 31) >> 5;
        const int t0 = lane * E;
        T v[EMAX];
#pragma unroll
        for (int j = 0; j < EMAX; j++) v[j] = (j < E && t0 + j < cl) ? in(rho + (t0 + j) * s) : ident;
#pragma unroll
        for (int j = 1; j < EMAX; j++) v[j] = op(v[j - 1], v[j]);
        T x = v[EMAX - 1];  // this lane's total (ident past its elements)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x = op(y, x);
        }
        T ex = __shfl_up_sync(FULL, x, 1);
        if (lane == 0) ex = ident;
#pragma unroll
        for (int j = 0; j < EMAX; j++)
            if (j < E && t0 + j < cl) out[rho + (t0 + j) * s] = op(ex, v[j]);
    }
    __syncthreads();
}

// Two strided prefix sums with the same stride in one pass (same scheme as
// warp_chains_scan): the two warp scans are independent, so each hides the
// other's shuffle latency.  Caller guarantees s < len and strided_by_warps.
template <class InA, class InB>
FS_D void warp_chains_scan2(InA ina, uint64_t* outa, InB inb, uint64_t* outb, int len, int s)
{
    constexpr int EMAX = 8;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int rho = threadIdx.x >> 5; rho < s; rho += nw) {
        const int cl = (len - 1 - rho) / s + 1;
        const int E = (cl + 31) >> 5;
        const int t0 = lane * E;
        uint64_t va[EMAX], vb[EMAX];
#pragma unroll
        for (int j = 0; j < EMAX; j++) {
            const bool ok = j < E && t0 + j < cl;
            const int p = rho + (t0 + j) * s;
            va[j] = ok ? ina(p) : 0ull;
            vb[j] = ok ? inb(p) : 0ull;
        }
#pragma unroll
        for (int j = 1; j < EMAX; j++) {
            va[j] += va[j - 1];
            vb[j] += vb[j - 1];
        }
        uint64_t x = va[EMAX - 1], y = vb[EMAX - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(FULL, x, o);
            const uint64_t v = __shfl_up_sync(FULL, y, o);
            if (lane >= o) {
                x += u;
                y += v;
            }
        }
        uint64_t ea = __shfl_up_sync(FULL, x, 1), eb = __shfl_up_sync(FULL, y, 1);
        if (lane == 0) ea = eb = 0;
#pragma unroll
        for (int j = 0; j < EMAX; j++)
            if (j < E && t0 + j < cl) {
                const int p = rho + (t0 + j) * s;
                outa[p] = ea + va[j];
                outb[p] = eb + vb[j];
            }
    }
    __syncthreads();
}

// Elements a thread of the segmented scans loads before it combines them: the
// loads of a segment are independent, the running sum is not.
constexpr int SCAN_BATCH = 8;

FS_D void block_strided_prefix_sum(const uint64_t* in, const Div32& dv_in, uint64_t* out, int len,
                                   int s, uint64_t* part)
{
    const int T = blockDim.x, tid = threadIdx.x;
    if (len <= 0) return;
    if (s < len && strided_by_warps(len, s)) {
        struct Add {
            FS_D uint64_t operator()(uint64_t a, uint64_t b) const { return a + b; }
        };
        warp_chains_scan<uint64_t>([&](int p) { return sps_in(in, p, dv_in); }, out, len, s, Add(),
                                   (uint64_t)0);
        return;
    }
    if (s >= T || s >= len) {
        // many short chains: one thread per chain
        int nch = s < len ? s : len;
        for (int rho = tid; rho < nch; rho += T) {
            uint64_t sum = 0;
            const int cl = (len - 1 - rho) / s + 1;
            for (int t = 0; t < cl; t += SCAN_BATCH) {
                uint64_t v[SCAN_BATCH];  // independent loads in flight
#pragma unroll
                for (int j = 0; j < SCAN_BATCH; j++) v[j] = t + j < cl ? sps_in(in, rho + (t + j) * s, dv_in) : 0;
#pragma unroll
                for (int j = 0; j < SCAN_BATCH; j++) {
                    sum += v[j];
                    if (t + j < cl) out[rho + (t + j) * s] = sum;
                }
            }
        }
        __syncthreads();
        return;
    }
    // s < T: chain rho = tid % s, segment g = tid / s, G segments per chain
    const int G = T / s;
    const int cl_max = (len - 1) / s + 1;  // longest chain (rho = 0)
    const int seg = (cl_max + G - 1) / G;
    const int rho = tid % s, g = tid / s;
    const bool act = g < G;
    const int t0 = g * seg;
    // this segment's elements t0 .. te-1 of chain rho (te <= t0: none)
    const int te = act ? min(t0 + seg, (len - 1 - rho) / s + 1) : t0;
    uint64_t sum = 0;
    for (int t = t0; t < te; t += SCAN_BATCH) {
        uint64_t v[SCAN_BATCH];
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) v[j] = t + j < te ? sps_in(in, rho + (t + j) * s, dv_in) : 0;
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) sum += v[j];
    }
    part[tid] = act ? sum : 0;
    __syncthreads();
    // inclusive scan along each chain: partials of chain rho sit at rho, rho+s, ...
    for (int off = s; off < G * s; off <<= 1) {
        uint64_t v = (act && tid >= off) ? part[tid - off] : 0;
        __syncthreads();
        if (act) part[tid] += v;
        __syncthreads();
    }
    uint64_t run = (act && g > 0) ? part[tid - s] : 0;  // exclusive prefix of this segment
    for (int t = t0; t < te; t += SCAN_BATCH) {
        uint64_t v[SCAN_BATCH];
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) v[j] = t + j < te ? sps_in(in, rho + (t + j) * s, dv_in) : 0;
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) {
            run += v[j];
            if (t + j < te) out[rho + (t + j) * s] = run;
        }
    }
    __syncthreads();
}

// Block-wide strided inclusive scan in place: x[p] = op(x[p - s], x[p]) for
// p = s..len-1, i.e. a running op along each residue class mod s (the same
// segmented scheme as block_strided_prefix_sum, for any associative op).
struct OpMin {
    template <class T>
    FS_D T operator()(T a, T b) const { return a < b ? a : b; }
};
struct OpMax {
    template <class T>
    FS_D T operator()(T a, T b) const { return a > b ? a : b; }
};
struct OpAdd {
    template <class T>
    FS_D T operator()(T a, T b) const { return a + b; }
};

template <class T, class Op>
FS_D void block_strided_scan(T* x, int len, int s, T* part, T ident, Op op)
{
    const int NT = blockDim.x, tid = threadIdx.x;
    if (len <= 0) return;
    if (s < len && strided_by_warps(len, s)) {
        warp_chains_scan<T>([&](int p) { return x[p]; }, x, len, s, op, ident);
        return;
    }
    if (s >= NT || s >= len) {
        const int nch = s < len ? s : len;
        for (int rho = tid; rho < nch; rho += NT) {
            T acc = ident;
            const int cl = (len - 1 - rho) / s + 1;
            for (int t = 0; t < cl; t += SCAN_BATCH) {
                T v[SCAN_BATCH];  // independent loads in flight
#pragma unroll
                for (int j = 0; j < SCAN_BATCH; j++) v[j] = t + j < cl ? x[rho + (t + j) * s] : ident;
#pragma unroll
                for (int j = 0; j < SCAN_BATCH; j++) {
                    acc = op(acc, v[j]);
                    if (t + j < cl) x[rho + (t + j) * s] = acc;
                }
            }
        }
        __syncthreads();
        return;
    }
    const int G = NT / s;
    const int cl_max = (len - 1) / s + 1;
    const int seg = (cl_max + G - 1) / G;
    const int rho = tid % s, g = tid / s;
    const bool act = g < G;
    const int t0 = g * seg;
    const int te = act ? min(t0 + seg, (len - 1 - rho) / s + 1) : t0;
    T acc = ident;
    for (int t = t0; t < te; t += SCAN_BATCH) {
        T v[SCAN_BATCH];
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) v[j] = t + j < te ? x[rho + (t + j) * s] : ident;
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) acc = op(acc, v[j]);
    }
    part[tid] = act ? acc : ident;
    __syncthreads();
    for (int off = s; off < G * s; off <<= 1) {
        const T v = (act && tid >= off) ? part[tid - off] : ident;
        __syncthreads();
        if (act) part[tid] = op(v, part[tid]);
        __syncthreads();
    }
    T run = (act && g > 0) ? part[tid - s] : ident;
    for (int t = t0; t < te; t += SCAN_BATCH) {
        T v[SCAN_BATCH];
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) v[j] = t + j < te ? x[rho + (t + j) * s] : ident;
#pragma unroll
        for (int j = 0; j < SCAN_BATCH; j++) {
            run = op(run, v[j]);
            if (t + j < te) x[rho + (t + j) * s] = run;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Run prefix, distributed over lanes: lane k (k < P-1) holds level k.
// ---------------------------------------------------------------------------
struct RunPrefix {
    int32_t a;  // a_k
    int32_t r;  // n - sum_{i <= k} a_i h_i
    int32_t l;  // sum_{i <= k} a_i
};

// Finds the leaf of lex rank `rank` from the leaf counts.  With
// W_k[p] = #{(a_k..a_{P-1}) : sum a_i h_i <= p}, the leaves under prefix
// (a_0..a_{k-1}) whose a_k is below x number W_k[p] - W_k[p - x h_k] (p the
// residual after level k-1), so a_k is the largest x with
// W_k[p - x h_k] >= W_k[p] - rank.  A 32-way search per level (lanes probe 32
// evenly spaced x).  Returns a_{P-1} (the index inside the run) and fills rp.
FS_D int32_t warp_unrank(const QueryConst& q, const int32_t* hs, const Div32* dvh,
                         const uint64_t* W, uint64_t rank, int lane, RunPrefix& rp)
{
    int32_t p = q.n;
    uint64_t rho = rank;
    int32_t lsum = 0;
    rp.a = 0;
    rp.r = q.n;
    rp.l = 0;
    const int np = q.P - 1;
    for (int k = 0; k < np; k++) {
        const uint64_t* Wk = W + (size_t)k * (size_t)(q.n + 1);
        const int32_t h = hs[k];
        const uint64_t top = Wk[p];
        const uint64_t target = top - rho;  // >= 1
        int32_t lo = 0, hi = (int32_t)div32((uint32_t)p, dvh[k]);
        while (lo < hi) {
            int32_t span = hi - lo + 1;
            int32_t step = (span + 31) >> 5;
            long long x = (long long)lo + (long long)lane * step;
            bool ok = false;
            if (x <= hi) ok = Wk[p - (int32_t)x * h] >= target;
            unsigned m = __ballot_sync(FULL, ok);
            if (m == 0) {  // cannot happen with exact tables; ends the search regardless
                hi = lo;
                break;
            }
            int j = 31 - __clz(m);
            lo = lo + j * step;
            hi = min(hi, lo + step - 1);
        }
        const int32_t a = lo;
        rho -= top - Wk[p - a * h];
        p -= a * h;
        lsum += a;
        if (lane == k) {
            rp.a = a;
            rp.r = p;
            rp.l = lsum;
        }
    }
    return (int32_t)rho;
}

// The same search by one thread: a binary search per level (about
// log2(p / h_k) probes), no warp cooperation.  A planner with many slices per
// warp spends a few instructions per slice this way instead of a few hundred.
// on_level(k, p, a) sees each prefix level k < P-1 with the residual p before
// it and its coordinate a; the run residual (after level P-2, n if P = 1) goes
// to p_run.  Returns a_{P-1}, the index inside the run.
template <class OnLevel>
FS_D int32_t thread_unrank(const QueryConst& q, const int32_t* hs, const Div32* dvh,
                           const uint64_t* W, uint64_t rank, int32_t& p_run, OnLevel on_level)
{
    int32_t p = q.n;
    uint64_t rho = rank;
    const int np = q.P - 1;
    for (int k = 0; k < np; k++) {
        const uint64_t* Wk = W + (size_t)k * (size_t)(q.n + 1);
        const int32_t h = hs[k];
        const uint64_t top = Wk[p];
        const uint64_t target = top - rho;  // >= 1
        // W_k[p - x h] >= target holds at lo and fails at hi (hi one past the range)
        int32_t lo = 0, hi = (int32_t)div32((uint32_t)p, dvh[k]) + 1;
        uint64_t wlo = top;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            const uint64_t w = Wk[p - mid * h];
            if (w >= target) {
                lo = mid;
                wlo = w;
            } else {
                hi = mid;
            }
        }
        rho -= top - wlo;
        on_level(k, p, lo);
        p -= lo * h;
    }
    p_run = p;
    return (int32_t)rho;
}

// Lex successor of the run prefix (levels 0..P-2): increment the deepest level
// that still fits and zero the levels below it.  Returns false if none.
FS_D bool warp_next_run(const QueryConst& q, int lane, int32_t hk, RunPrefix& rp)
{
    const int np = q.P - 1;
    bool can = (lane < np) && (rp.r >= hk);
    unsigned m = __ballot_sync(FULL, can);
    if (m == 0) return false;
    int k = 31 - __clz(m);
    int32_t nr = __shfl_sync(FULL, rp.r - hk, k);
    int32_t nl = __shfl_sync(FULL, rp.l + 1, k);
    if (lane == k) {
        rp.a += 1;
        rp.r = nr;
        rp.l = nl;
    } else if (lane > k && lane < np) {
        rp.a = 0;
        rp.r = nr;
        rp.l = nl;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Slice start states, written once per call by the planner (k_plan): per slice
// START_W int32, [k] = a_k of the run prefix (k < P-1) and [START_W-1] = the
// index of the slice's first leaf inside its run (-1 for an empty slice).
// ---------------------------------------------------------------------------
constexpr int START_W = FS_MAX_D;

// Loads slice s's start into the lane-distributed run prefix; returns the
// index of the first leaf inside its run.
FS_D int32_t warp_load_start(const QueryConst& q, const int32_t* hs, const int32_t* starts,
                             uint64_t s, int lane, RunPrefix& rp)
{
    const int np = q.P - 1;
    const int32_t* st = starts + s * START_W;
    const int32_t a = lane < np ? st[lane] : 0;
    const int32_t b = st[START_W - 1];
    int32_t ph = lane < np ? a * hs[lane] : 0;
    int32_t pl = a;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int32_t t1 = __shfl_up_sync(FULL, ph, o);
        const int32_t t2 = __shfl_up_sync(FULL, pl, o);
        if (lane >= o) {
            ph += t1;
            pl += t2;
        }
    }
    rp.a = a;
    rp.r = q.n - ph;
    rp.l = pl;
    return b;
}

// ---------------------------------------------------------------------------
// The slice walk.  A run is the sequence of leaves a_{P-1} = b, b+1, ... under
// one prefix of levels 0..P-2 (residual R; leaf a has residual R - a h_{P-1}).
// Runs that differ only in level P-2 ("siblings") are taken 32 at a time: lane
// j holds sibling j, so the lex successor of the prefix (a ballot over the
// levels) runs once per group of siblings.  Lane j works out which of run j's
// leaves the slice takes (a warp scan of the run lengths) and which of those
// are visited (common-divisor skipping), then the warp visits the group's leaves
// 32 per step in one of two ways (walk_slice_packed, walk_slice_lex_packed).
// Cons must provide
//   static constexpr bool ANY_ORDER -- the consumer does not depend on the
//                                    order of the leaves (counts, lengths,
//                                    predicates): full 32-leaf steps run by run,
//                                    then the runs' remainders packed; else the
//                                    group's leaves packed in lex order
//   static constexpr int UNROLL   -- full 32-leaf steps per loop trip (ANY_ORDER)
//   static constexpr bool SKIP    -- visit only the leaves that common-divisor
//                                    skipping keeps (for consumers whose per-leaf
//                                    work outweighs the per-run class arithmetic)
//   void group_begin(const QueryConst&, const RunPrefix& rp, int lane,
//                    int32_t ac, int32_t lpc)
//       -- a sibling group starts (warp-uniform): levels 0..P-3 are rp.a on
//          lanes 0..P-3; its runs have level P-2 = ac + j and prefix sum lpc + j
//   bool chunk(const QueryConst&, int lane, bool valid, int32_t r, int32_t a,
//              int32_t lp)
//       -- one leaf per lane: residual r left for the pair, a = a_{P-1},
//          lp = sum of the leaf's run prefix (so its run is lp - lpc siblings
//          into the group); invalid lanes must not use r; returns true to stop
//          the walk (warp-uniform);
//   void fault() -- the slice ran past the last leaf (a planner fault).
// Returns true if the consumer stopped the walk.
// ---------------------------------------------------------------------------
// Common-divisor skipping for one run: of the leaves a = b .. b+nh-1 of a
// run with residual R, only a = first + k ma (k < cnt) can have completions
// (QueryConst::sk_*); cnt = 0 when R is not a multiple of sk_g.
FS_D void skip_class(const QueryConst& q, uint32_t R, uint32_t b, uint32_t nh, uint32_t& first,
                     uint32_t& cnt, uint32_t& ma)
{
    const uint32_t Rg = div32(R, q.dv_skg[0]);
    if (Rg * (uint32_t)q.sk_g[0] != R) {
        cnt = 0;
        return;
    }
    const uint32_t m = (uint32_t)q.sk_m[0];
    ma = m;
    if (m == 1) return;  // every leaf of the run qualifies
    const uint32_t rs = Rg - div32(Rg, q.dv_skm[0]) * m;  // Rg mod m
    uint32_t as;                                          // the class: rs * inv mod m
    if (m < 46341u) {  // the product stays below 2^31, the range of div32
        const uint32_t p = rs * (uint32_t)q.sk_inv[0];
        as = p - div32(p, q.dv_skm[0]) * m;
    } else {
        as = (uint32_t)(((uint64_t)rs * (uint64_t)(uint32_t)q.sk_inv[0]) % m);
    }
    const uint32_t bm = b - div32(b, q.dv_skm[0]) * m;  // b mod m
    const uint32_t off = as >= bm ? as - bm : as + m - bm;
    first = b + off;
    cnt = off < nh ? div32(nh - 1 - off, q.dv_skm[0]) + 1 : 0;
}

// Issue slots a warp step costs in each way through a sibling group, for the
// choice in walk_slice_packed: a step over one run's 32 leaves (residual and
// coordinate advanced once per step), a step with each lane on its own run,
// a packed step (plus the 5-step search for each lane's run and the shuffles
// of its run's data), and each run's turn in the full-step loop.
// Cons::CHUNK_OPS estimates the consumer's per-leaf work.  The constants were
// set from the measured walks of both kinds on the heavy count query (long
// runs of a few dozen visited leaves: lanes) and the single large query
// (slices of a few hundred leaves: packed).
// Cons::R_INDEXED says it reads a shared 32-bit table at the residual itself:
// lanes whose residuals are k apart then meet 2^ctz(k)-way bank conflicts
// (k = hsib for lanes on sibling runs, k = the step between visited leaves
// for lanes on one run), each extra way costing about a few issue slots.
template <class Cons>
struct WalkCost {
    static constexpr uint32_t full = Cons::CHUNK_OPS + 4;
    static constexpr uint32_t lane = Cons::CHUNK_OPS + 3;
    static constexpr uint32_t pack = Cons::CHUNK_OPS + 36;
    static constexpr uint32_t per_run = 12;  // a run's turn in the full-step loop
    static constexpr uint32_t per_way = 4;
};

FS_D uint32_t conflict_ways(uint32_t stride)
{
    return stride == 0 ? 32u : 1u << min(5, __ffs(stride) - 1);
}

// Whether a consumer wants each sibling group's visited-leaf total before the
// group is walked (Cons::group_leaves(uint32_t), warp-uniform, below 2^31).
template <class C, class = void>
struct HasGroupLeaves {
    static constexpr bool value = false;
};
template <class C>
struct HasGroupLeaves<C, decltype((void)&C::group_leaves)> {
    static constexpr bool value = true;
};
// Whether a consumer walks with staggered lanes (Cons::STAG, below): a
// per-launch choice, so that consumers that do not stagger keep their code.
template <class C, class = void>
struct Staggers {
    static constexpr bool value = false;
};
template <class C>
struct Staggers<C, decltype((void)C::STAG)> {
    static constexpr bool value = C::STAG;
};
// Whether a consumer wants to hear when a group is done (Cons::group_end()).
template <class C, class = void>
struct HasGroupEnd {
    static constexpr bool value = false;
};
template <class C>
struct HasGroupEnd<C, decltype((void)&C::group_end)> {
    static constexpr bool value = true;
};

// The walk for consumers that do not depend on the order of the leaves inside
// a slice (Cons::ANY_ORDER: counts, length statistics, predicates).  A group of
// up to 32 sibling runs is taken in one of two ways, chosen per group from the
// runs' visited-leaf counts cnt_j (q.walk can force either):
//  - lanes: lane j walks run j by itself, all lanes stepping together until the
//    longest run is done (max cnt_j steps; a lane whose run is done idles);
//  - packed: each run's full 32-leaf steps run by run (lane l takes the run's
//    leaves l, l + 32, ..), then the remainders of all runs (fewer than 32
//    leaves each) packed into shared steps, lane l of such a step finding its
//    run by a 5-step search over the runs' offsets (sum_j floor(cnt_j / 32)
//    full steps and ceil(sum_j (cnt_j mod 32) / 32) packed ones).
// Sibling runs differ in length by about hsib / h_in leaves per lane, so when
// runs are a few dozen leaves long the lanes way wastes little and avoids the
// packed steps' search; with long runs or few siblings the packed way wins.
// The per-run bookkeeping is done once per group by all lanes together.
template <class Cons>
FS_D bool walk_slice_packed(const QueryConst& q, const int32_t* hs, const Div32* dvh,
                            const int32_t* starts, uint64_t s, uint64_t nleaves, int lane,
                            int32_t hk, Cons& cons)
{
    RunPrefix rp;
    int32_t b = warp_load_start(q, hs, starts, s, lane, rp);
    const int np = q.P - 1;
    const uint32_t hin = (uint32_t)hs[np];
    const bool skip = Cons::SKIP && (q.sk_m[0] > 1 || q.sk_g[0] > 1);
    const uint32_t ma = skip ? (uint32_t)q.sk_m[0] : 1u;  // step of a between visited leaves
    const uint32_t mstep = ma * hin;
    // every run has fewer than 2^26 leaves: a group's leaf total fits 31 bits
    const bool small_runs = div32((uint32_t)q.n, q.dv_in) < (1u << 26) - 1;
    const uint32_t hsib = np > 0 ? (uint32_t)hs[np - 1] : 0u;
    uint64_t rem = nleaves;
    for (;;) {
        // The group: lane j holds run j of the next runs in lex order.  Runs
        // that differ only at level P-2 (a sibling set) have residuals hsib
        // apart and prefix sums one apart; a consumer that needs only each
        // lane's own run (Cons::MULTI_SET) lets the lanes after a set that
        // ends early take the next sets whole, up to 32 runs or the slice's
        // end.  `cur` ends as the prefix of the group's last set.
        RunPrefix cur = rp;
        uint32_t Rj = 0, bj = 0, left = 0;
        int32_t lpj = 0;
        uint32_t filled = 0, base_last = 0;
        int32_t Rc = q.n, lpc = 0, ac = 0;
        for (;;) {
            uint32_t nsib = 1;
            if (np > 0) {
                Rc = __shfl_sync(FULL, cur.r, np - 1);
                lpc = __shfl_sync(FULL, cur.l, np - 1);
                ac = __shfl_sync(FULL, cur.a, np - 1);
                nsib = div32((uint32_t)Rc, dvh[np - 1]) + 1;
            }
            if (nsib > 32 - filled) nsib = 32 - filled;
            const uint32_t j = (uint32_t)lane - filled;  // wraps for the lanes before
            if (j < nsib) {
                Rj = (uint32_t)Rc - j * hsib;
                lpj = lpc + (int32_t)j;
                bj = (filled == 0 && j == 0) ? (uint32_t)b : 0u;
                left = div32(Rj, q.dv_in) + 1 - bj;
            }
            base_last = filled;
            filled += nsib;
            if (!Cons::MULTI_SET || !small_runs || np == 0 || filled >= 32) break;
            // the slice ends inside the lanes filled so far
            if ((uint64_t)__reduce_add_sync(FULL, left) >= rem) break;
            // the next set, the successor of this set's last run, joins only
            // if it fits whole: small sets share a group, and a large set keeps
            // its own groups (a set's first runs are its longest, its last its
            // shortest, so a group cut across two sets would be uneven)
            RunPrefix nxt = cur;
            if (lane == np - 1) {
                nxt.a = ac + (int32_t)nsib - 1;
                nxt.r = (int32_t)((uint32_t)Rc - (nsib - 1) * hsib);
                nxt.l = lpc + (int32_t)nsib - 1;
            }
            if (!warp_next_run(q, lane, hk, nxt)) break;  // no runs left (the walk's own check follows)
            const uint32_t nnext = div32((uint32_t)__shfl_sync(FULL, nxt.r, np - 1), dvh[np - 1]) + 1;
            if (nnext > 32 - filled) break;
            cur = nxt;
        }
        const bool act = (uint32_t)lane < filled;
        uint32_t ns, nh;  // runs taken; leaves of run j in the slice
        uint64_t took;    // leaves of the runs taken
        const uint32_t gsum = small_runs ? __reduce_add_sync(FULL, left) : 0u;
        if (small_runs && (uint64_t)gsum <= rem) {
            // the whole group lies in the slice (the common case)
            ns = filled;
            nh = left;
            took = gsum;
        } else {
            uint64_t ir = left;  // leaves of runs 0..j
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t t = __shfl_up_sync(FULL, ir, o);
                if (lane >= o) ir += t;
            }
            // take the runs whose leaves so far stay below 2^31 (at least one),
            // so the visited-leaf offsets below fit 32 bits
            ns = __popc(__ballot_sync(FULL, act && ir < (1ull << 31)));
            if (ns == 0) ns = 1;
            const uint64_t er = ir - left;
            nh = 0;
            if ((uint32_t)lane < ns && er < rem) nh = rem - er < (uint64_t)left ? (uint32_t)(rem - er) : left;
            took = __shfl_sync(FULL, ir, (int)ns - 1);
        }
        uint32_t first = bj, cnt = nh, mj = 1;
        if (skip && nh > 0) skip_class(q, Rj, bj, nh, first, cnt, mj);
        const uint32_t nfull = cnt >> 5, part = cnt & 31;
        cons.group_begin(q, cur, lane, ac, lpc);  // single-set groups: their set
        if constexpr (HasGroupLeaves<Cons>::value) cons.group_leaves(__reduce_add_sync(FULL, cnt));
        const uint32_t mxc = __reduce_max_sync(FULL, cnt);
        // Lanes on sibling runs read a residual-indexed table at addresses
        // hsib apart: 2^ctz(hsib)-way bank conflicts.  With an odd step between
        // a run's leaves, holding lane j back j >> (5 - ctz(hsib)) steps puts
        // the lanes' residuals in 32 different banks at every step, for
        // 2^ctz(hsib) - 1 extra steps per group (stag: consumers launched with
        // Cons::STAG, for queries where it applies; the lanes way only).
        const uint32_t wsib = Cons::R_INDEXED ? conflict_ways(hsib) : 1u;
        const bool stag = Staggers<Cons>::value && hsib != 0 && wsib > 1 && (mstep & 1u);
        bool lanes = q.walk == FS_WALK_LANES;
        if (q.walk == FS_WALK_AUTO) {
            const uint32_t sfull = __reduce_add_sync(FULL, nfull);
            const uint32_t spart = __reduce_add_sync(FULL, part);
            const uint32_t rfull = __popc(__ballot_sync(FULL, nfull > 0));
            using C = WalkCost<Cons>;
            uint32_t cl = C::lane, cf = C::full, cp = C::pack, xl = 0;
            if (Cons::R_INDEXED) {
                if (stag)
                    xl = wsib - 1;
                else
                    cl += (wsib - 1) * C::per_way;
                cf += (conflict_ways(mstep) - 1) * C::per_way;
                cp += C::per_way;  // lanes on mixed runs: about two ways
            }
            lanes = (uint64_t)(mxc + xl) * cl <= (uint64_t)sfull * cf + (uint64_t)rfull * C::per_run +
                                                     (uint64_t)((spart + 31) >> 5) * cp;
        }
        if (lanes) {
            // lane j: run j's visited leaves a = first + k ma, k < cnt, leaf k
            // at step i = k + dl (dl: the lane's delay, 0 unless stag); while
            // every lane has started and none has ended the bound check is
            // left out
            const uint32_t dl = stag ? (uint32_t)lane >> (5 - (__ffs(wsib) - 1)) : 0u;
            uint32_t a = first - dl * ma, r = Rj - first * hin + dl * mstep;
            const int32_t lp = lpj;
            const uint32_t e = cnt + dl;                        // one past the lane's last step
            const uint32_t lo_u = stag ? wsib - 1 : 0u;         // every lane has started
            const uint32_t hi_u = __reduce_min_sync(FULL, e);   // none has ended
            const uint32_t mxe = stag ? __reduce_max_sync(FULL, e) : mxc;
            uint32_t i = 0;
            if (Staggers<Cons>::value) {
                for (const uint32_t p1 = min(lo_u, mxe); i < p1; i++) {
                    if (cons.chunk(q, lane, i - dl < cnt, (int32_t)r, (int32_t)a, lp)) return true;
                    r -= mstep;
                    a += ma;
                }
            }
            if (Cons::UNROLL > 1) {
                for (; i + Cons::UNROLL <= hi_u; i += Cons::UNROLL) {
#pragma unroll
                    for (int u = 0; u < Cons::UNROLL; u++) {
                        if (cons.chunk(q, lane, true, (int32_t)r, (int32_t)a, lp)) return true;
                        r -= mstep;
                        a += ma;
                    }
                }
            }
            for (; i < hi_u; i++) {
                if (cons.chunk(q, lane, true, (int32_t)r, (int32_t)a, lp)) return true;
                r -= mstep;
                a += ma;
            }
            for (; i < mxe; i++) {
                if (cons.chunk(q, lane, i - dl < cnt, (int32_t)r, (int32_t)a, lp)) return true;
                r -= mstep;
                a += ma;
            }
        } else {
            // the full steps, run by run: lane l takes the run's leaves l, l + 32, ..
            for (uint32_t m = __ballot_sync(FULL, nfull > 0); m; m &= m - 1) {
                const int j = __ffs(m) - 1;
                const uint32_t nf = __shfl_sync(FULL, nfull, j);
                uint32_t a = __shfl_sync(FULL, first, j) + (uint32_t)lane * ma;
                uint32_t r = __shfl_sync(FULL, Rj, j) - a * hin;
                const int32_t lp = __shfl_sync(FULL, lpj, j);
                uint32_t i = 0;
                if (Cons::UNROLL > 1) {
                    for (; i + Cons::UNROLL <= nf; i += Cons::UNROLL) {
#pragma unroll
                        for (int u = 0; u < Cons::UNROLL; u++) {
                            if (cons.chunk(q, lane, true, (int32_t)r, (int32_t)a, lp)) return true;
                            r -= 32u * mstep;
                            a += 32u * ma;
                        }
                    }
                }
                for (; i < nf; i++) {
                    if (cons.chunk(q, lane, true, (int32_t)r, (int32_t)a, lp)) return true;
                    r -= 32u * mstep;
                    a += 32u * ma;
                }
            }
            // the remainders, packed: run j's last `part` visited leaves
            const uint32_t pa = first + (cnt - part) * ma;  // the first of them
            const uint32_t r0 = Rj - pa * hin;
            uint32_t iv = part;  // remainder leaves of runs 0..j
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, iv, o);
                if (lane >= o) iv += t;
            }
            const uint32_t ev = iv - part;
            const uint32_t tot = __shfl_sync(FULL, iv, 31);
            for (uint32_t t0 = 0; t0 < tot; t0 += 32) {
                const uint32_t t = t0 + (uint32_t)lane;
                // the run of visited leaf t: the last j with ev_j <= t (runs past
                // the group's end have ev_j = tot)
                int j = 0;
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const uint32_t e = __shfl_sync(FULL, ev, j + st);
                    if (e <= t) j += st;
                }
                const uint32_t k = t - __shfl_sync(FULL, ev, j);
                const uint32_t a = __shfl_sync(FULL, pa, j) + k * ma;
                const uint32_t r = __shfl_sync(FULL, r0, j) - k * mstep;
                const int32_t lp = __shfl_sync(FULL, lpj, j);
                if (cons.chunk(q, lane, t < tot, (int32_t)r, (int32_t)a, lp)) return true;
            }
        }
        if constexpr (HasGroupEnd<Cons>::value) cons.group_end();
        if (took >= rem) return false;
        rem -= took;
        b = 0;
        // the last run taken becomes the current one (it is in the last set:
        // a group that ends early ends the slice); step to its lex successor
        if (np == 0) {
            cons.fault();  // the slice claims leaves past the last one
            return false;
        }
        const uint32_t jl = ns - 1 - base_last;
        if (lane == np - 1) {
            cur.a = ac + (int32_t)jl;
            cur.r = (int32_t)((uint32_t)Rc - jl * hsib);
            cur.l = lpc + (int32_t)jl;
        }
        rp = cur;
        if (!warp_next_run(q, lane, hk, rp)) {
            cons.fault();
            return false;
        }
    }
}

// The walk in lex order with the leaves of a sibling group packed (for a
// consumer that needs the order: enumerate): the warp steps through the
// group's visited leaves 32 at a time in lex order, whatever run each belongs
// to; lane l finds the run of its leaf by a 5-step search over the runs'
// offsets.  cons.group_begin(q, rp, lane, ac, lpc) starts each group (its runs
// have level P-2 = ac + j and prefix sum lpc + j, j = 0, 1, ..); chunk gets
// each lane's own a and lp.
template <class Cons>
FS_D bool walk_slice_lex_packed(const QueryConst& q, const int32_t* hs, const Div32* dvh,
                                const int32_t* starts, uint64_t s, uint64_t nleaves, int lane,
                                int32_t hk, Cons& cons)
{
    RunPrefix rp;
    int32_t b = warp_load_start(q, hs, starts, s, lane, rp);
    const int np = q.P - 1;
    const uint32_t hin = (uint32_t)hs[np];
    const bool skip = Cons::SKIP && (q.sk_m[0] > 1 || q.sk_g[0] > 1);
    const uint32_t ma = skip ? (uint32_t)q.sk_m[0] : 1u;
    const uint32_t mstep = ma * hin;
    uint64_t rem = nleaves;
    for (;;) {
        int32_t Rc = q.n, lpc = 0, ac = 0;
        uint32_t hsib = 0, nsib = 1;
        if (np > 0) {
            Rc = __shfl_sync(FULL, rp.r, np - 1);
            lpc = __shfl_sync(FULL, rp.l, np - 1);
            ac = __shfl_sync(FULL, rp.a, np - 1);
            hsib = (uint32_t)hs[np - 1];
            nsib = div32((uint32_t)Rc, dvh[np - 1]) + 1;
            if (nsib > 32) nsib = 32;
        }
        const bool act = (uint32_t)lane < nsib;
        const uint32_t Rj = (uint32_t)Rc - (uint32_t)lane * hsib;
        const uint32_t bj = lane == 0 ? (uint32_t)b : 0u;
        const uint32_t left = act ? div32(Rj, q.dv_in) + 1 - bj : 0u;
        uint64_t ir = left;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, ir, o);
            if (lane >= o) ir += t;
        }
        uint32_t ns = __popc(__ballot_sync(FULL, act && ir < (1ull << 31)));
        if (ns == 0) ns = 1;
        const uint64_t er = ir - left;
        uint32_t nh = 0;
        if ((uint32_t)lane < ns && er < rem) nh = rem - er < (uint64_t)left ? (uint32_t)(rem - er) : left;
        uint32_t first = bj, cnt = nh, mj = 1;
        if (skip && nh > 0) skip_class(q, Rj, bj, nh, first, cnt, mj);
        uint32_t iv = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, iv, o);
            if (lane >= o) iv += t;
        }
        const uint32_t ev = iv - cnt;
        const uint32_t tot = __shfl_sync(FULL, iv, 31);
        const uint32_t r0 = Rj - first * hin;
        cons.group_begin(q, rp, lane, ac, lpc);
        for (uint32_t t0 = 0; t0 < tot; t0 += 32) {
            const uint32_t t = t0 + (uint32_t)lane;
            int j = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const uint32_t e = __shfl_sync(FULL, ev, j + st);
                if (e <= t) j += st;
            }
            const uint32_t k = t - __shfl_sync(FULL, ev, j);
            const uint32_t a = __shfl_sync(FULL, first, j) + k * ma;
            const uint32_t r = __shfl_sync(FULL, r0, j) - k * mstep;
            if (cons.chunk(q, lane, t < tot, (int32_t)r, (int32_t)a, lpc + j)) return true;
        }
        const uint64_t took = __shfl_sync(FULL, ir, (int)ns - 1);
        if (took >= rem) return false;
        rem -= took;
        b = 0;
        if (np == 0) {
            cons.fault();
            return false;
        }
        if (lane == np - 1) {
            rp.a = ac + (int32_t)ns - 1;
            rp.r = (int32_t)((uint32_t)Rc - (ns - 1) * hsib);
            rp.l = lpc + (int32_t)ns - 1;
        }
        if (!warp_next_run(q, lane, hk, rp)) {
            cons.fault();
            return false;
        }
    }
}

template <class Cons>
FS_D bool walk_slice(const QueryConst& q, const int32_t* hs, const Div32* dvh,
                     const int32_t* starts, uint64_t s, uint64_t nleaves, int lane, int32_t hk,
                     Cons& cons)
{
    if constexpr (Cons::ANY_ORDER)
        return walk_slice_packed(q, hs, dvh, starts, s, nleaves, lane, hk, cons);
    else
        return walk_slice_lex_packed(q, hs, dvh, starts, s, nleaves, lane, hk, cons);
}

// ---------------------------------------------------------------------------
// The same slice counted run by run: T3[p] (the trailing-three table of q:
// the factorizations of p over levels P-1, P, P+1) is the count of all leaves
// of a run from residual p downwards, so a run segment a_{P-1} = b .. b+m-1
// with run residual R holds T3[R - b h] - T3[R - (b+m) h] factorizations
// (the second term 0 when the segment reaches the run's end).  Lane j takes
// sibling run j; the warp advances 32 runs per step instead of 32 leaves.
// Returns this lane's part of the slice count (the caller sums the warp);
// *fault is set if the slice claims leaves past the last one.
// ---------------------------------------------------------------------------
// rp, b: the slice's start (run prefix in the lanes, index in the first run);
// T3 in global or shared memory.
FS_D uint64_t slice_count_runs(const QueryConst& q, const int32_t* hs, const Div32* dvh,
                               RunPrefix rp, int32_t b, uint64_t nleaves, int lane, int32_t hk,
                               const uint64_t* T3, bool* fault)
{
    const int np = q.P - 1;
    const int32_t hin = hs[np];
    uint64_t rem = nleaves;
    uint64_t acc = 0;
    for (;;) {
        int32_t Rc = q.n, ac = 0;
        uint32_t hsib = 0, nsib = 1;
        if (np > 0) {
            Rc = __shfl_sync(FULL, rp.r, np - 1);
            ac = __shfl_sync(FULL, rp.a, np - 1);
            hsib = (uint32_t)hs[np - 1];
            nsib = div32((uint32_t)Rc, dvh[np - 1]) + 1;
            if (nsib > 32) nsib = 32;
        }
        const bool act = (uint32_t)lane < nsib;
        const int32_t R = (int32_t)((uint32_t)Rc - (uint32_t)lane * hsib);
        const int32_t bj = lane == 0 ? b : 0;
        // leaves this run still has (from bj on), and how many of them the slice takes
        const uint64_t len = act ? (uint64_t)(div32((uint32_t)R, q.dv_in) + 1 - (uint32_t)bj) : 0;
        uint64_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const uint64_t excl = incl - len;
        const uint64_t m = excl >= rem ? 0 : (rem - excl < len ? rem - excl : len);
        if (m > 0) {
            const int32_t r0 = R - bj * hin;
            const int32_t r1 = r0 - (int32_t)m * hin;
            acc += T3[r0] - (r1 >= 0 ? T3[r1] : 0ull);
        }
        const uint64_t tot = __shfl_sync(FULL, incl, 31);
        if (tot >= rem) return acc;
        rem -= tot;
        b = 0;
        if (np == 0) {
            *fault = true;
            return acc;
        }
        if (lane == np - 1) {
            rp.a = ac + (int32_t)nsib - 1;
            rp.r = (int32_t)((uint32_t)Rc - (nsib - 1) * hsib);
            rp.l = 0;
        }
        if (!warp_next_run(q, lane, hk, rp)) {
            *fault = true;
            return acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-block copies of the dynamically indexed per-level constants, the slice
// queue loop, and the device error flag.
// ---------------------------------------------------------------------------
struct SmemQ {
    int32_t h[FS_MAX_D];
    int32_t col[FS_MAX_D];
    Div32 dvh[FS_MAX_D];
    SliceSplit split;  // the planner's split (planned_split)
};

// The block's copy of the query constants and of the planner's split (ctr: the
// call's counters, written by the planner before this kernel).  The caller
// synchronises the block before using sq.
FS_D void load_smemq(const QueryConst& q, SmemQ& sq, const uint64_t* ctr)
{
    const int t = threadIdx.x;
    if (t < FS_MAX_D) {
        sq.h[t] = q.h[t];
        sq.col[t] = q.col[t];
        sq.dvh[t] = q.dv_h[t];
    }
    if (t == FS_MAX_D) sq.split = planned_split(ctr);
}

// Walk slices with `cons`.  The planner (k_plan) has written the number of
// slices, the number of leaves and each slice's start state.  Warp w of the
// grid takes slice w first (no atomic: every warp starting at once on one
// counter would serialise at L2), then pops slices W, W+1, ... (W = warps in
// the grid) from the queue counter, one slice ahead so the atomic's latency
// overlaps the walk.
template <class Cons>
FS_D void run_queue(const QueryConst& q, const SmemQ& sq, const Scratch& sc, int queue, Cons& cons)
{
    const int lane = threadIdx.x & 31;
    const int32_t hk = lane < q.P - 1 ? sq.h[lane] : 0;
    const uint64_t S_all = sc.ctr[CTR_SEFF];
    const uint64_t S = sc.s_hi < S_all ? sc.s_hi : S_all;  // the window's slices
    const uint64_t W = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long* qc = (unsigned long long*)&sc.ctr[queue];
    unsigned long long s = sc.s_lo + (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    while (s < S) {
        unsigned long long nxt = 0;
        if (lane == 0) nxt = sc.s_lo + atomicAdd(qc, 1ull) + W;
        const uint64_t k0 = sq.split.start(s), k1 = sq.split.start(s + 1);
        cons.slice_begin(q, s);
        bool stop = false;
        if (k1 > k0) stop = walk_slice(q, sq.h, sq.dvh, sc.starts, s, k1 - k0, lane, hk, cons);
        cons.slice_end(q, s);
        if (stop) break;
        s = __shfl_sync(FULL, nxt, 0);
    }
}

// Whether any warp of this block takes a slice in run_queue: its first warp's
// static slice s_lo + (global warp index) is inside the window, or every later
// warp's is not either (and the dynamic ones start past all warps).  Lets a
// block skip its prologue (a shared-memory table copy) when the planner chose
// fewer slices than the grid has warps.
FS_D bool block_has_slices(const Scratch& sc)
{
    const uint64_t S_all = sc.ctr[CTR_SEFF];
    const uint64_t S = sc.s_hi < S_all ? sc.s_hi : S_all;
    return sc.s_lo + (uint64_t)blockIdx.x * (blockDim.x >> 5) < S;
}

// Called by thread 0 of every block of a count walk after it has added its
// part to ctr[CTR_COUNT]: the last block to finish copies the total to
// *dev_count (the caller's device memory), so no separate copy kernel runs.
FS_D void publish_count(uint64_t* ctr, uint64_t* dev_count)
{
    if (!dev_count) return;
    __threadfence();  // this block's addition is visible before its ticket
    const unsigned long long t = atomicAdd((unsigned long long*)&ctr[CTR_DONE], 1ull);
    if (t == gridDim.x - 1) {
        __threadfence();
        *dev_count = atomicAdd((unsigned long long*)&ctr[CTR_COUNT], 0ull);
    }
}

// The first output row of slice s (see Scratch::blk).
FS_D uint64_t slice_row0(const Scratch& sc, uint64_t s)
{
    return sc.slice_off[s] + (sc.blk ? sc.blk[s / SLICE_GROUP] : 0ull);
}

// Offsets of slices counted group by group (SLICE_GROUP slices, counts in
// shared memory cnt[]): writes each slice of group grp its offset within the
// group (slice_off) and the group total (blk[grp]); the block that finishes
// the last of the ngroups groups (ticket in ctr[CTR_DONE]) turns blk into
// exclusive group offsets and writes the total to ctr[CTR_TOTAL] and
// *dev_count.  Called by every thread of a 1024-thread block; wsum: 32 shared
// words; last: a shared flag.
FS_D void group_offsets(const Scratch& sc, const uint64_t* cnt, uint64_t grp, uint32_t ngroups,
                        uint64_t S, uint64_t* dev_count, uint64_t* wsum, bool* last)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t g0 = grp * SLICE_GROUP;
    uint64_t v = tid < SLICE_GROUP ? cnt[tid] : 0, x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (tid < SLICE_GROUP) {
        uint64_t before = 0;
        for (int k = 0; k < w; k++) before += wsum[k];
        if (g0 + tid < S) sc.slice_off[g0 + tid] = before + x - v;
    }
    if (tid == 0) {
        uint64_t tot = 0;
        for (int k = 0; k < SLICE_GROUP / 32; k++) tot += wsum[k];
        sc.blk[grp] = tot;
        __threadfence();  // the total is visible before the ticket
        const unsigned long long t = atomicAdd((unsigned long long*)&sc.ctr[CTR_DONE], 1ull);
        *last = t == ngroups - 1;
    }
    __syncthreads();
    if (!*last) return;
    // the last group: exclusive scan of the group totals (in place), the total
    __threadfence();
    const uint32_t nb = ngroups;
    uint64_t carry = 0;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t i = base + tid;
        const uint64_t y0 = i < nb ? *(volatile uint64_t*)&sc.blk[i] : 0;
        uint64_t y = y0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += t;
        }
        __syncthreads();  // wsum is free
        if (lane == 31) wsum[w] = y;
        __syncthreads();
        if (w == 0) {
            uint64_t z = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t t = __shfl_up_sync(FULL, z, o);
                if (lane >= o) z += t;
            }
            wsum[lane] = z;
        }
        __syncthreads();
        if (i < nb) sc.blk[i] = carry + (w > 0 ? wsum[w - 1] : 0) + y - y0;
        carry += wsum[31];
    }
    __syncthreads();
    if (tid == 0) {
        // the end of the last slice: row offset S = the total
        if (S % SLICE_GROUP == 0) sc.blk[S / SLICE_GROUP] = carry;
        sc.slice_off[S] = carry - sc.blk[S / SLICE_GROUP];
        sc.ctr[CTR_TOTAL] = carry;
        if (dev_count) *dev_count = carry;
    }
}

// Sets the device error flag the host checks after a synchronous call.
FS_D void flag_fault(uint64_t* ctr)
{
    if ((threadIdx.x & 31) == 0) atomicOr((unsigned long long*)&ctr[CTR_ERR], 1ull);
}

// ---------------------------------------------------------------------------
// The pair (A, B) at a leaf with residual r: the solutions x A + y B = r with
// x, y >= 0 are x = x0 + t v, y = y0 - t u for 0 <= t < c.  (Sec. 3.2.4: after
// a valid candidate the next valid value of a_{d-1} is v = B / gcd(A, B)
// steps lower; here the walk jumps straight to the valid values.)
//
// Table path (lcm(A,B) small): with r = q lcm + w, 0 <= w < lcm, the class of
// x mod v and the first solution depend on w only:
//   E[w] = -1 if G does not divide w, else [w >= x0(w) A];  c = q + E[w]
//   X0[w] = x0(w) (-1 if G does not divide w);  YD[w] = (w - x0 A) / B;
//   y0 = q u + YD[w].
// General path: the same quantities by division.
// ---------------------------------------------------------------------------
// The smallest x of the pair's solutions from t = (r / G) mod v: t u^-1 mod v.
// Below v = 46341 the product t inv < v^2 stays under 2^31 and the remainder
// is one invariant division; above, a 64-bit remainder.
template <class QC>
FS_D uint32_t pair_x0(const QC& q, uint32_t t)
{
    if (q.v < 46341) {
        const uint32_t pr = t * (uint32_t)q.inv;
        return pr - div32(pr, q.dv_v) * (uint32_t)q.v;
    }
    return (uint32_t)(((uint64_t)t * (uint32_t)q.inv) % (uint32_t)q.v);
}

template <bool TAB, class QC>
FS_D uint32_t pair_count(const QC& q, const int8_t* E, int32_t r)
{
    if (TAB) {
        uint32_t qq = div32((uint32_t)r, q.dv_lcm);
        int32_t w = r - (int32_t)(qq * q.lcm);
        int32_t e = E[w];
        return e < 0 ? 0u : qq + (uint32_t)e;
    } else {
        uint32_t rg = div32((uint32_t)r, q.dv_G);
        if ((int32_t)rg * q.G != r) return 0u;
        uint32_t t = rg - div32(rg, q.dv_v) * (uint32_t)q.v;
        uint32_t x0 = pair_x0(q, t);
        uint32_t xmax = div32((uint32_t)r, q.dv_A);
        return xmax >= x0 ? div32(xmax - x0, q.dv_v) + 1u : 0u;
    }
}

template <bool TAB, class QC>
FS_D uint32_t pair_xy(const QC& q, const int32_t* X0, const int32_t* YD, int32_t r, int32_t& x0,
                      int32_t& y0)
{
    if (TAB) {
        uint32_t qq = div32((uint32_t)r, q.dv_lcm);
        int32_t w = r - (int32_t)(qq * q.lcm);
        int32_t xx = X0[w];
        if (xx < 0) return 0u;
        int32_t yd = YD[w];
        x0 = xx;
        y0 = (int32_t)qq * q.u + yd;
        return qq + (yd >= 0 ? 1u : 0u);
    } else {
        uint32_t rg = div32((uint32_t)r, q.dv_G);
        if ((int32_t)rg * q.G != r) return 0u;
        uint32_t t = rg - div32(rg, q.dv_v) * (uint32_t)q.v;
        uint32_t xx = pair_x0(q, t);
        uint32_t xmax = div32((uint32_t)r, q.dv_A);
        if (xmax < xx) return 0u;
        x0 = (int32_t)xx;
        y0 = (int32_t)div32((uint32_t)(r - (int32_t)xx * q.A), q.dv_B);
        return div32(xmax - xx, q.dv_v) + 1u;
    }
}

// The pair tables for w = start, start + stride, ... < lcm (see pair_count):
// E[w] = -1 if G does not divide w, else [w >= x0(w) A]; X0[w] = x0(w) or -1;
// YD[w] = (w - x0(w) A) / B.  Null table pointers are skipped.
FS_D void pair_tables_fill(const QueryConst& q, int8_t* E, int32_t* X0, int32_t* YD,
                           uint32_t start, uint32_t stride)
{
    for (uint32_t w = start; w < q.lcm; w += stride) {
        int8_t e = -1;
        int32_t x0 = -1, yd = 0;
        if (w % (uint32_t)q.G == 0) {
            const uint64_t wg = w / (uint32_t)q.G;
            const uint64_t x = ((wg % (uint64_t)q.v) * (uint64_t)q.inv) % (uint64_t)q.v;
            const int64_t rest = (int64_t)w - (int64_t)x * q.A;  // divisible by B
            x0 = (int32_t)x;
            yd = (int32_t)(rest / q.B);
            e = rest >= 0 ? 1 : 0;
        }
        if (E) E[w] = e;
        if (X0) X0[w] = x0;
        if (YD) YD[w] = yd;
    }
}

// The pair constants alone, for consumers that keep them in registers while
// the rest of the query's constants live in shared or global memory.
struct PairC {
    Div32 dv_lcm, dv_A, dv_B, dv_G, dv_v;
    uint32_t lcm;
    int32_t A, B, G, u, v, inv, delta;
};

FS_D PairC pair_consts(const QueryConst& q)
{
    PairC p;
    p.dv_lcm = q.dv_lcm;
    p.dv_A = q.dv_A;
    p.dv_B = q.dv_B;
    p.dv_G = q.dv_G;
    p.dv_v = q.dv_v;
    p.lcm = q.lcm;
    p.A = q.A;
    p.B = q.B;
    p.G = q.G;
    p.u = q.u;
    p.v = q.v;
    p.inv = q.inv;
    p.delta = q.delta;
    return p;
}

// The trailing-k tables of q (k = 3 or 4) for p = 0..n, built by the calling
// block (any size; part64 / part32 hold blockDim.x entries).  Level P-1 is
// summed over the pair's closed form; each further level (P-2 for k = 4) is
// one more strided scan of the same tables in place (the TRAIL roles of
// k_precompute).  Any of T, MN, MX may be NULL: k_precompute builds each on a
// block of its own.
// tmax (nullable, global): receives the largest entry of T (atomicMax).
FS_D void trailing_tables_block(const QueryConst& q, int k, uint64_t* T, int32_t* MN, int32_t* MX,
                                uint64_t* part64, int32_t* part32, uint64_t* tmax = nullptr)
{
    const int len = q.n + 1;
    const bool lens = MN || MX;
    for (int lvl = q.P - 1; lvl >= q.P + 2 - k; lvl--) {
        const int h = q.h[lvl];
        const Div32 dvh = q.dv_h[lvl];
        for (int p = threadIdx.x; p < len; p += blockDim.x) {
            const int32_t t = (int32_t)div32((uint32_t)p, dvh);
            if (lvl == q.P - 1 && !lens) {
                T[p] = pair_count<false>(q, (const int8_t*)nullptr, p);
            } else if (lvl == q.P - 1) {
                int32_t x0 = 0, y0 = 0;
                const uint32_t c =
                    pair_xy<false>(q, (const int32_t*)nullptr, (const int32_t*)nullptr, p, x0, y0);
                if (T) T[p] = c;
                const int32_t l0 = x0 + y0, l1 = l0 + (int32_t)(c - 1) * q.delta;
                if (MN) MN[p] = (c > 0 ? min(l0, l1) : TRIPLE_NONE) - t;
                if (MX) MX[p] = (c > 0 ? max(l0, l1) : -TRIPLE_NONE) - t;
            } else {
                if (MN) MN[p] -= t;
                if (MX) MX[p] -= t;
            }
        }
        __syncthreads();
        if (T) block_strided_scan<uint64_t>(T, len, h, part64, (uint64_t)0, OpAdd());
        if (MN) block_strided_scan<int32_t>(MN, len, h, part32, (int32_t)TRIPLE_NONE, OpMin());
        if (MX) block_strided_scan<int32_t>(MX, len, h, part32, (int32_t)-TRIPLE_NONE, OpMax());
        if (lens) {
            for (int p = threadIdx.x; p < len; p += blockDim.x) {
                const int32_t t = (int32_t)div32((uint32_t)p, dvh);
                if (MN) MN[p] += t;
                if (MX) MX[p] += t;
            }
        }
        __syncthreads();
    }
    if (tmax && T) {
        uint64_t m = 0;
        for (int p = threadIdx.x; p < len; p += blockDim.x) m = T[p] > m ? T[p] : m;
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t y = __shfl_xor_sync(FULL, m, o);
            m = y > m ? y : m;
        }
        if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)tmax, (unsigned long long)m);
    }
}

// The query the trailing-k walk runs over: k - 2 prefix levels fewer (in place).
FS_HD void reduce_to_trailing(QueryConst& r, int k)
{
    r.sk_g[0] = r.sk_g[k - 2];
    r.sk_m[0] = r.sk_m[k - 2];
    r.sk_inv[0] = r.sk_inv[k - 2];
    r.dv_skg[0] = r.dv_skg[k - 2];
    r.dv_skm[0] = r.dv_skm[k - 2];
    r.D -= k - 2;
    r.P -= k - 2;
    r.dv_in = r.dv_h[r.P - 1];
    r.nw = r.P - 1;
    r.tab_e = 0;
    r.tab_xy = 0;
    r.lcm = 0;
}

// warp sums
FS_D uint64_t warp_sum_u64(uint64_t v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

}  // namespace fsi
