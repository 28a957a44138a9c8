// The PAIR method: bounded lexicographic walk over the leaves, with the last
// two coordinates of every leaf resolved in closed form (the congruence step
// of Sec. 3.2.4 taken to its end).  Persistent warps pop slices from a device
// queue (Sec. 4: each worker owns a bounded slice of the lex order), and each
// warp walks 32 leaves per step (walk.cuh).  Consumers (Sec. 2): count, length
// statistics, predicate, save (enumerate).
#include "launch.h"
#include "walk.cuh"

namespace fsi {

// ===========================================================================
// count
// ===========================================================================
// The count of a leaf with residual r = qq lcm + w is qq + E[w], E[w] in
// {0, 1} for every w the walk visits (its residual is a multiple of G by
// common-divisor skipping; E[w] = -1 marks the other classes).  The table path
// keeps E as a bitmask, one 32-bit word per 32 classes, with every word
// repeated 32 times so that lane l reads its own copy at bank l: the lanes'
// lookups at scattered w never meet in a bank (4 lcm bytes, 64 KB at most).
// ACC32: a lane sums its counts of one sibling group in 32 bits and adds
// them to its 64-bit total when the group is done (QueryConst::acc32 bounds
// that sum).  FDIV: the quotient by lcm is one multiply-high
// (QueryConst::fdiv).
template <bool TAB, bool PER_SLICE, bool ACC32, bool FDIV = false>
struct CountCons {
    const uint32_t* Eb;  // TAB: the replicated bitmask
    uint64_t* slice_cnt;
    uint64_t acc;    // this lane, current slice
    uint64_t total;  // this lane, all slices
    uint32_t acc32;  // this lane, current group (ACC32)
    uint64_t* ctr;
    static constexpr int UNROLL = 8;  // full steps per loop trip (4: 1.5 % slower)
    static constexpr bool SKIP = true;
    static constexpr bool ANY_ORDER = true;
    static constexpr bool MULTI_SET = true;
    static constexpr uint32_t CHUNK_OPS = 10;
    static constexpr bool R_INDEXED = false;
    FS_D void fault() { flag_fault(ctr); }
    FS_D void group_begin(const QueryConst&, const RunPrefix&, int, int32_t, int32_t) {}
    FS_D void group_end()
    {
        if (ACC32) {
            acc += acc32;
            acc32 = 0;
        }
    }
    FS_D void slice_begin(const QueryConst&, uint64_t) {}
    FS_D void slice_end(const QueryConst&, uint64_t s)
    {
        if (PER_SLICE) {
            uint64_t v = warp_sum_u64(acc);
            if ((threadIdx.x & 31) == 0) slice_cnt[s] = v;
        }
        total += acc;
        acc = 0;
    }
    FS_D bool chunk(const QueryConst& q, int lane, bool valid, int32_t r, int32_t, int32_t)
    {
        if (valid) {
            uint32_t c;
            if (TAB) {
                const uint32_t qq = FDIV ? __umulhi((uint32_t)r, q.lcm_m1) : div32((uint32_t)r, q.dv_lcm);
                const uint32_t w = (uint32_t)r - qq * q.lcm;
                const uint32_t m = Eb[(w & ~31u) | (uint32_t)lane];
                c = qq + (__funnelshift_r(m, m, w) & 1u);
            } else {
                c = pair_count<false>(q, (const int8_t*)nullptr, r);
            }
            if (ACC32)
                acc32 += c;
            else
                acc += c;
        }
        return false;
    }
};

// The replicated bitmask of E (see CountCons) from the byte table, by a block:
// word k holds bit i = [E[32 k + i] > 0].
FS_D void build_count_bitmask(const int8_t* E, uint32_t lcm, uint32_t* Eb)
{
    const uint32_t lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const uint32_t words = (lcm + 31) >> 5;
    for (uint32_t k = threadIdx.x >> 5; k < words; k += nw) {
        const uint32_t w = k * 32 + lane;
        const uint32_t m = __ballot_sync(FULL, w < lcm && E[w] > 0);
        Eb[k * 32 + lane] = m;
    }
}

template <bool TAB, bool PER_SLICE, bool ACC32, bool FDIV = false>
__global__ void __launch_bounds__(256) k_pair_count(const __grid_constant__ QueryConst q,
                                                    Scratch sc, int queue, uint64_t* dev_count)
{
    __shared__ SmemQ sq;
    __shared__ unsigned long long bsum;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq, sc.ctr);
    if (threadIdx.x == 0) bsum = 0;
    uint32_t* Eb = (uint32_t*)dyn;
    if (TAB) build_count_bitmask(sc.E, q.lcm, Eb);
    __syncthreads();
    CountCons<TAB, PER_SLICE, ACC32, FDIV> cons{Eb, sc.slice_cnt, 0, 0, 0u, sc.ctr};
    run_queue(q, sq, sc, queue, cons);
    uint64_t v = warp_sum_u64(cons.total);
    if ((threadIdx.x & 31) == 0) atomicAdd(&bsum, (unsigned long long)v);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long*)&sc.ctr[CTR_COUNT], bsum);
        publish_count(sc.ctr, dev_count);
    }
}

// ===========================================================================
// length statistics: count, min, max and the histogram of sum a_i
// ===========================================================================
// Along a leaf the lengths are l0 + t * delta, t = 0..c-1, an arithmetic
// progression; it is added to the histogram as a strided difference array
// (+1 at its low end, -1 one stride past its high end), finalised by a
// stride-|delta| prefix sum.
template <bool TAB>
struct LenCons {
    const int32_t* X0;
    const int32_t* YD;
    unsigned long long* Dh;
    int32_t s;
    uint64_t cnt;
    uint32_t mn, mx;
    uint64_t* ctr;
    static constexpr int UNROLL = 2;
    static constexpr bool SKIP = true;
    static constexpr bool ANY_ORDER = true;
    static constexpr bool MULTI_SET = true;
    static constexpr uint32_t CHUNK_OPS = 30;
    static constexpr bool R_INDEXED = false;
    FS_D void fault() { flag_fault(ctr); }
    FS_D void group_begin(const QueryConst&, const RunPrefix&, int, int32_t, int32_t) {}
    FS_D void slice_begin(const QueryConst&, uint64_t) {}
    FS_D void slice_end(const QueryConst&, uint64_t) {}
    FS_D bool chunk(const QueryConst& q, int, bool valid, int32_t r, int32_t a, int32_t lp)
    {
        if (valid) {
            int32_t x0 = 0, y0 = 0;
            uint32_t c = pair_xy<TAB>(q, X0, YD, r, x0, y0);
            if (c > 0) {
                cnt += c;
                int32_t l0 = lp + a + x0 + y0;
                int32_t lt = l0 + (int32_t)(c - 1) * q.delta;
                int32_t lo = min(l0, lt), hi = max(l0, lt);
                mn = min(mn, (uint32_t)lo);
                mx = max(mx, (uint32_t)hi);
                if (s == 0) {
                    atomicAdd(&Dh[lo], (unsigned long long)c);
                } else {
                    atomicAdd(&Dh[lo], 1ull);
                    atomicAdd(&Dh[hi + s], ~0ull);  // -1 modulo 2^64
                }
            }
        }
        return false;
    }
};

template <bool TAB, bool SMEMD>
__global__ void __launch_bounds__(256) k_pair_len(const __grid_constant__ QueryConst q,
                                                  Scratch sc, int queue)
{
    __shared__ SmemQ sq;
    __shared__ unsigned long long bsum;
    __shared__ unsigned int bmin, bmax;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq, sc.ctr);
    if (threadIdx.x == 0) {
        bsum = 0;
        bmin = 0xffffffffu;
        bmax = 0;
    }
    unsigned char* p = dyn;
    unsigned long long* Dh = (unsigned long long*)sc.D;
    if (SMEMD) {
        Dh = (unsigned long long*)p;
        for (int i = threadIdx.x; i < q.dbins; i += blockDim.x) Dh[i] = 0;
        p += (size_t)q.dbins * 8;
    }
    int32_t* X0 = (int32_t*)p;
    int32_t* YD = X0 + (TAB ? q.lcm : 0);
    if (TAB)
        for (uint32_t i = threadIdx.x; i < q.lcm; i += blockDim.x) {
            X0[i] = sc.X0[i];
            YD[i] = sc.YD[i];
        }
    __syncthreads();
    const int32_t s = q.delta < 0 ? -q.delta : q.delta;
    LenCons<TAB> cons{X0, YD, Dh, s, 0, 0xffffffffu, 0, sc.ctr};
    run_queue(q, sq, sc, queue, cons);
    uint64_t v = warp_sum_u64(cons.cnt);
    uint32_t mn = cons.mn, mx = cons.mx;
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(FULL, mn, o));
        mx = max(mx, __shfl_xor_sync(FULL, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&bsum, (unsigned long long)v);
        atomicMin(&bmin, mn);
        atomicMax(&bmax, mx);
    }
    __syncthreads();
    if (threadIdx.x == 0 && bsum > 0) {
        atomicAdd((unsigned long long*)&sc.ctr[CTR_COUNT], bsum);
        atomicMax((unsigned long long*)&sc.ctr[CTR_MINC], (unsigned long long)(0xffffffffu - bmin));
        atomicMax((unsigned long long*)&sc.ctr[CTR_MAX], (unsigned long long)bmax);
    }
    if (SMEMD) {
        for (int i = threadIdx.x; i < q.dbins; i += blockDim.x)
            if (Dh[i]) atomicAdd((unsigned long long*)&sc.D[i], Dh[i]);
    }
}

// ===========================================================================
// length histogram: one difference array per warp, in shared memory
// ===========================================================================
// With r = qq lcm + w, the pair's solutions at a leaf have lengths (beyond the
// leaf's own prefix length lpa = lp + a) from e0 = L0[w] + qq u to
// e1 = L1[w] + qq v in steps of delta, where L0 = X0 + YD and
// L1 = L0 + (E - 1) delta (E = [YD >= 0]; c = qq + E solutions).  The
// difference array takes +1 at the lower end and -1 one step s = |delta| past
// the upper end: lo = lpa + TL[w].x + qq clo and hp = lpa + TL[w].y + qq chp,
// (clo, chp) = (v, u) when delta < 0 (e1 is the lower end), (u, v) when
// delta > 0.  Then hp - lo = c s, so a leaf has solutions iff lo < hp.  Every
// leaf the walk visits has a residual divisible by G (common-divisor
// skipping), so w always has solutions in its class; the bound check on hp
// only keeps a wrong index from reaching memory.
//
// Each warp adds into its own 32-bit array (lanes of one warp may still meet
// on a bin, hence the shared-memory atomics); a bin of it changes by at most
// one per visited leaf, so a warp flushes its array into the global 64-bit one
// before 2^31 leaves have been added to it, and the block sums its warps'
// arrays into the global one at the end.  The count, the minimum and the
// maximum come from the finished histogram (k_len_finalize).  FDIV: the
// quotient by lcm is one multiply-high (QueryConst::fdiv).
template <bool FDIV>
struct HistCons {
    const int2* TL;
    uint32_t* Dw;  // this warp's difference array (wrapping 32-bit)
    uint64_t* Dg;  // the global difference array (wrapping 64-bit)
    int32_t clo, chp;
    uint32_t dbins;
    uint32_t since;  // visited leaves added to Dw since it was last flushed (warp-uniform)
    uint64_t* ctr;
    static constexpr int UNROLL = 2;
    static constexpr bool SKIP = true;
    static constexpr bool ANY_ORDER = true;
    static constexpr bool MULTI_SET = true;
    static constexpr uint32_t CHUNK_OPS = 14;
    static constexpr bool R_INDEXED = false;
    FS_D void fault() { flag_fault(ctr); }
    FS_D void group_begin(const QueryConst&, const RunPrefix&, int, int32_t, int32_t) {}
    FS_D void flush()
    {
        __syncwarp();
        for (uint32_t i = threadIdx.x & 31; i < dbins; i += 32) {
            const uint32_t v = Dw[i];
            if (v) {
                atomicAdd((unsigned long long*)&Dg[i], (unsigned long long)(int64_t)(int32_t)v);
                Dw[i] = 0;
            }
        }
        __syncwarp();
    }
    // the walk announces the visited leaves of each sibling group before it
    // takes them (warp-uniform, fewer than 2^31)
    FS_D void group_leaves(uint32_t tot)
    {
        if (since + tot >= 0x80000000u) {
            flush();
            since = 0;
        }
        since += tot;
    }
    FS_D void slice_begin(const QueryConst&, uint64_t) {}
    FS_D void slice_end(const QueryConst&, uint64_t) {}
    FS_D bool chunk(const QueryConst& q, int, bool valid, int32_t r, int32_t a, int32_t lp)
    {
        if (valid) {
            const uint32_t qq = FDIV ? __umulhi((uint32_t)r, q.lcm_m1) : div32((uint32_t)r, q.dv_lcm);
            const int32_t w = r - (int32_t)(qq * q.lcm);
            const int2 t = TL[w];
            const int32_t lpa = lp + a;
            const int32_t lo = lpa + t.x + (int32_t)qq * clo;
            const int32_t hp = lpa + t.y + (int32_t)qq * chp;
            if ((uint32_t)lo < (uint32_t)hp && (uint32_t)hp < dbins) {
                atomicAdd(&Dw[lo], 1u);
                atomicAdd(&Dw[hp], 0xffffffffu);  // -1 modulo 2^32
            }
        }
        return false;
    }
};

// Per-warp 32-bit arrays (dbins rounded up to 32 words each) and the packed
// endpoint table (lcm int2) in dynamic shared memory.
static int hist_smem_bytes(const QueryConst& q, int threads)
{
    return (int)q.lcm * 8 + (threads / 32) * ((q.dbins + 31) & ~31) * 4;
}

template <bool FDIV>
__global__ void __launch_bounds__(256) k_pair_hist(const __grid_constant__ QueryConst q,
                                                   Scratch sc, int queue)
{
    __shared__ SmemQ sq;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq, sc.ctr);
    const int nwarps = blockDim.x >> 5, wid = threadIdx.x >> 5;
    int2* TL = (int2*)dyn;
    uint32_t* D0 = (uint32_t*)(TL + q.lcm);
    const int dstride = (q.dbins + 31) & ~31;
    for (int i = threadIdx.x; i < dstride * nwarps; i += blockDim.x) D0[i] = 0;
    const int32_t s = q.delta < 0 ? -q.delta : q.delta;
    for (uint32_t w = threadIdx.x; w < q.lcm; w += blockDim.x) {
        const int32_t x0 = sc.X0[w], yd = sc.YD[w];
        int2 t = make_int2(1, 0);  // no solutions in this class (never visited)
        if (x0 >= 0) {
            const int32_t L0 = x0 + yd, L1 = yd >= 0 ? L0 : L0 - q.delta;
            t = q.delta < 0 ? make_int2(L1, L0 + s) : make_int2(L0, L1 + s);
        }
        TL[w] = t;
    }
    __syncthreads();
    HistCons<FDIV> cons{TL,      D0 + wid * dstride, sc.D, q.delta < 0 ? q.v : q.u, q.delta < 0 ? q.u : q.v,
                  (uint32_t)q.dbins, 0u, sc.ctr};
    run_queue(q, sq, sc, queue, cons);
    __syncthreads();
    // the block's warp arrays, summed, into the global array
    for (int i = threadIdx.x; i < q.dbins; i += blockDim.x) {
        int64_t v = 0;
        for (int k = 0; k < nwarps; k++) v += (int32_t)D0[k * dstride + i];
        if (v) atomicAdd((unsigned long long*)&sc.D[i], (unsigned long long)v);
    }
}

// ===========================================================================
// any: does some factorization satisfy the linear predicate?
// ===========================================================================
// Along a leaf the predicate's linear form is V0 + t * dw (t = 0..c-1), so each
// leaf is decided in closed form: an equality is a divisibility test, an
// inequality compares the two ends, a congruence is a linear congruence in t.
FS_D bool pred_on_progression(const PredConst& pc, int64_t V0, uint32_t c)
{
    const int64_t dw = pc.dw;
    if (pc.modulus > 0) {
        const int64_t M = pc.modulus;
        int64_t diff = (pc.c - V0) % M;
        if (diff < 0) diff += M;
        if (diff % pc.gM != 0) return false;
        uint64_t t0 = ((uint64_t)(diff / pc.gM) * (uint64_t)pc.invq) % (uint64_t)pc.Mq;
        return t0 < (uint64_t)c;
    }
    if (pc.op == 0) {
        if (dw == 0) return V0 == pc.c;
        int64_t diff = pc.c - V0;
        if (diff % dw != 0) return false;
        int64_t t = diff / dw;
        return t >= 0 && t < (int64_t)c;
    }
    int64_t Vl = V0 + (int64_t)(c - 1) * dw;
    if (pc.op == 1) return min(V0, Vl) <= pc.c;
    return max(V0, Vl) >= pc.c;
}

template <bool TAB>
struct AnyCons {
    const int32_t* X0;
    const int32_t* YD;
    const PredConst* pc;
    unsigned long long* flag;
    int64_t pwb;  // weighted sum of the sibling group's first run prefix
    int32_t lpb;  // its prefix sum (a lane's run is lp - lpb runs further)
    int poll;
    uint64_t* ctr;
    static constexpr int UNROLL = 1;
    static constexpr bool SKIP = true;
    static constexpr bool ANY_ORDER = true;
    static constexpr bool MULTI_SET = false;
    static constexpr uint32_t CHUNK_OPS = 30;
    static constexpr bool R_INDEXED = false;
    FS_D void fault() { flag_fault(ctr); }
    FS_D void group_begin(const QueryConst& q, const RunPrefix& rp, int lane, int32_t ac, int32_t lpc)
    {
        int64_t v = (lane < q.P - 2) ? pc->w[lane] * (int64_t)rp.a : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        pwb = v + (q.P >= 2 ? pc->w[q.P - 2] * (int64_t)ac : 0);
        lpb = lpc;
    }
    FS_D void slice_begin(const QueryConst&, uint64_t) {}
    FS_D void slice_end(const QueryConst&, uint64_t) {}
    FS_D bool chunk(const QueryConst& q, int lane, bool valid, int32_t r, int32_t a, int32_t lp)
    {
        bool f = false;
        if (valid) {
            int32_t x0 = 0, y0 = 0;
            uint32_t c = pair_xy<TAB>(q, X0, YD, r, x0, y0);
            if (c > 0) {
                const int64_t pw = pwb + (q.P >= 2 ? pc->w[q.P - 2] * (int64_t)(lp - lpb) : 0);
                int64_t V0 = pw + pc->w[q.P - 1] * (int64_t)a +
                             pc->w[q.P] * (int64_t)x0 + pc->w[q.P + 1] * (int64_t)y0;
                f = pred_on_progression(*pc, V0, c);
            }
        }
        if (__any_sync(FULL, f)) {
            if (lane == 0) atomicExch(flag, 1ull);
            return true;
        }
        if (++poll >= 64) {
            poll = 0;
            unsigned long long g = 0;
            if (lane == 0) g = *(volatile unsigned long long*)flag;
            g = __shfl_sync(FULL, g, 0);
            if (g) return true;
        }
        return false;
    }
};

template <bool TAB>
__global__ void __launch_bounds__(256, 4) k_pair_any(const __grid_constant__ QueryConst q,
                                                  Scratch sc, int queue,
                                                  const __grid_constant__ PredConst pred)
{
    __shared__ SmemQ sq;
    __shared__ PredConst spc;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq, sc.ctr);
    if (threadIdx.x == 0) spc = pred;
    int32_t* X0 = (int32_t*)dyn;
    int32_t* YD = X0 + (TAB ? q.lcm : 0);
    if (TAB)
        for (uint32_t i = threadIdx.x; i < q.lcm; i += blockDim.x) {
            X0[i] = sc.X0[i];
            YD[i] = sc.YD[i];
        }
    __syncthreads();
    AnyCons<TAB> cons{X0, YD, &spc, (unsigned long long*)&sc.ctr[CTR_FOUND], 0, 0, 0, sc.ctr};
    run_queue(q, sq, sc, queue, cons);
}

// ===========================================================================
// TRIPLE: the trailing three coordinates from tables (Sec. 6.1)
// ===========================================================================
// The walk runs over the prefixes of the first D-3 levels (the reduced query
// q3 has one prefix level fewer); the leaf with residual r contributes
// T3[r] factorizations with lengths lp + a + [MN3[r], MX3[r]].
// MODE 0: the count; 1: count, minimum and maximum length; 2: minimum and
// maximum only.  With SMEMT the length range comes from a shared-memory table
// MM packing MN3[r] (low 16 bits, 0xffff: no completion) and MX3[r] (high 16
// bits) per residual (MODE 2 always).
template <int MODE, bool PER_SLICE, bool SMEMT, bool STAG_ = false>
struct TripleCons {
    const uint64_t* T3;
    const uint32_t* T32;  // SMEMT: shared-memory uint32 copy of T3, or NULL
    const uint32_t* MM;   // SMEMT, MODE 1 / 2: the packed length range in shared memory
    const int32_t* MN3;
    const int32_t* MX3;
    uint64_t* slice_cnt;
    uint64_t* ctr;
    uint64_t acc, total;
    int32_t mn, mx;
    static constexpr int UNROLL = 4;
    static constexpr bool SKIP = false;
    static constexpr bool ANY_ORDER = true;
    static constexpr bool MULTI_SET = true;
    static constexpr uint32_t CHUNK_OPS = MODE == 1 ? 12 : MODE == 2 ? 6 : 4;
    static constexpr bool R_INDEXED = true;
    static constexpr bool STAG = STAG_;  // staggered lanes (walk_slice_packed)
    FS_D void fault() { flag_fault(ctr); }
    FS_D void group_begin(const QueryConst&, const RunPrefix&, int, int32_t, int32_t) {}
    FS_D void slice_begin(const QueryConst&, uint64_t) {}
    FS_D void slice_end(const QueryConst&, uint64_t s)
    {
        if (PER_SLICE) {
            const uint64_t v = warp_sum_u64(acc);
            if ((threadIdx.x & 31) == 0) slice_cnt[s] = v;
        }
        total += acc;
        acc = 0;
    }
    FS_D bool chunk(const QueryConst&, int, bool valid, int32_t r, int32_t a, int32_t lp)
    {
        if (MODE == 2) {
            if (valid) {
                const uint32_t v = MM[r];
                const int32_t lo = (int32_t)(v & 0xffffu);
                if (lo != 0xffff) {
                    mn = min(mn, lp + a + lo);
                    mx = max(mx, lp + a + (int32_t)(v >> 16));
                }
            }
            return false;
        }
        if (valid) {
            uint64_t c;
            if constexpr (SMEMT)
                c = T32 ? (uint64_t)T32[r] : __ldg(&T3[r]);
            else
                c = __ldg(&T3[r]);
            acc += c;
            if (MODE && c) {
                if constexpr (SMEMT) {
                    const uint32_t v = MM[r];
                    mn = min(mn, lp + a + (int32_t)(v & 0xffffu));
                    mx = max(mx, lp + a + (int32_t)(v >> 16));
                } else {
                    mn = min(mn, lp + a + __ldg(&MN3[r]));
                    mx = max(mx, lp + a + __ldg(&MX3[r]));
                }
            }
        }
        return false;
    }
};

// SMEMT: the count table is copied to shared memory as uint32 (when its
// largest entry, recorded by the precompute, fits), so the lookups of the walk
// hit shared memory instead of L2; for MODE 2 the packed length range.
template <int MODE, bool PER_SLICE, bool SMEMT, bool STAG = false>
__global__ void __launch_bounds__(SMEMT ? 1024 : 256, SMEMT ? 1 : 4) k_triple_walk(
    const __grid_constant__ QueryConst q3, Scratch sc, int queue, const uint64_t* T3,
    const int32_t* MN3, const int32_t* MX3, uint64_t* dev_count)
{
    __shared__ SmemQ sq;
    __shared__ unsigned long long bsum;
    __shared__ int bmin, bmax;
    extern __shared__ __align__(16) unsigned char dyn[];
    if (!block_has_slices(sc)) {  // skips the table copy too
        if (threadIdx.x == 0) publish_count(sc.ctr, dev_count);
        return;
    }
    load_smemq(q3, sq, sc.ctr);
    if (threadIdx.x == 0) {
        bsum = 0;
        bmin = 0x7fffffff;
        bmax = -1;
    }
    uint32_t* T32 = nullptr;
    uint32_t* MM = nullptr;
    const uint32_t len = (uint32_t)q3.n + 1;
    if (SMEMT && MODE) {  // MODE 1: after the count table; MODE 2: alone
        MM = (uint32_t*)dyn + (MODE == 1 ? len : 0);
        for (uint32_t p = threadIdx.x; p < len; p += blockDim.x) {
            const int32_t lo = __ldg(&MN3[p]), hi = __ldg(&MX3[p]);
            MM[p] = lo >= 0xffff ? 0xffffu : (uint32_t)lo | ((uint32_t)hi << 16);
        }
    }
    if (SMEMT && MODE != 2 && sc.ctr[CTR_TMAX] <= 0xffffffffull) {
        T32 = (uint32_t*)dyn;
        const uint32_t bd = blockDim.x;
        for (uint32_t p = threadIdx.x; p < len; p += 4 * bd) {  // four loads in flight
            uint64_t v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] = p + k * bd < len ? __ldg(&T3[p + k * bd]) : 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (p + k * bd < len) T32[p + k * bd] = (uint32_t)v[k];
        }
    }
    __syncthreads();
    TripleCons<MODE, PER_SLICE, SMEMT, STAG> cons{T3, T32, MM, MN3, MX3, sc.slice_cnt, sc.ctr, 0, 0, 0x7fffffff, -1};
    run_queue(q3, sq, sc, queue, cons);
    const uint64_t v = warp_sum_u64(cons.total);
    int mn = cons.mn, mx = cons.mx;
    if (MODE)
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(FULL, mn, o));
            mx = max(mx, __shfl_xor_sync(FULL, mx, o));
        }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&bsum, (unsigned long long)v);
        if (MODE) {
            atomicMin(&bmin, mn);
            atomicMax(&bmax, mx);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (MODE == 2 && bmax >= 0) {
            atomicMax((unsigned long long*)&sc.ctr[CTR_MINC], (unsigned long long)(0xffffffffu - (uint32_t)bmin));
            atomicMax((unsigned long long*)&sc.ctr[CTR_MAX], (unsigned long long)(uint32_t)bmax);
        } else if (MODE != 2 && bsum > 0) {
            atomicAdd((unsigned long long*)&sc.ctr[CTR_COUNT], bsum);
            if (MODE) {
                atomicMax((unsigned long long*)&sc.ctr[CTR_MINC], (unsigned long long)(0xffffffffu - (uint32_t)bmin));
                atomicMax((unsigned long long*)&sc.ctr[CTR_MAX], (unsigned long long)(uint32_t)bmax);
            }
        }
        publish_count(sc.ctr, dev_count);
    }
}

// Per-slice counts of PAIR slices from the trailing-three table, run by run
// (slice_count_runs): the first walk of fs_enumerate when the table is cheap.
// Block b counts the SLICE_GROUP slices from b * SLICE_GROUP on (each warp 8
// consecutive ones) and group_offsets turns the counts into row offsets, so
// no separate scan over all slices runs.
__global__ void __launch_bounds__(1024) k_pair_slice_runs(const __grid_constant__ QueryConst q,
                                                          Scratch sc, const uint64_t* T3,
                                                          uint64_t* dev_count)
{
    __shared__ SmemQ sq;
    __shared__ uint64_t cnt[SLICE_GROUP];
    __shared__ uint64_t wsum[32];
    __shared__ bool last;
    load_smemq(q, sq, sc.ctr);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t hk = lane < q.P - 1 ? sq.h[lane] : 0;
    const uint64_t S = sc.ctr[CTR_SEFF];
    const SliceSplit split = sq.split;
    bool fault = false;
    constexpr int PER_WARP = SLICE_GROUP / 32;
    for (int i = 0; i < PER_WARP; i++) {
        const uint64_t s = (uint64_t)blockIdx.x * SLICE_GROUP + w * PER_WARP + i;
        uint64_t c = 0;
        if (s < S) {
            const uint64_t k0 = split.start(s), k1 = split.start(s + 1);
            if (k1 > k0) {
                RunPrefix rp;
                const int32_t b = warp_load_start(q, sq.h, sc.starts, s, lane, rp);
                c = slice_count_runs(q, sq.h, sq.dvh, rp, b, k1 - k0, lane, hk, T3, &fault);
            }
        }
        c = warp_sum_u64(c);
        if (lane == 0) {
            cnt[w * PER_WARP + i] = c;
            if (s < S) sc.slice_cnt[s] = c;
        }
    }
    if (__any_sync(FULL, fault)) flag_fault(sc.ctr);
    __syncthreads();
    group_offsets(sc, cnt, blockIdx.x, gridDim.x, S, dev_count, wsum, &last);
}

cudaError_t launch_pair_slice_runs(const QueryConst& q, const Scratch& sc, const uint64_t* T3,
                                   uint64_t S_req, uint64_t* dev_count, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((S_req + SLICE_GROUP - 1) / SLICE_GROUP);
    k_pair_slice_runs<<<blocks, 1024, 0, st>>>(q, sc, T3, dev_count);
    return cudaGetLastError();
}

// The planner and enumerate's slice offsets in one launch, with no walk: the
// factorizations before a lex position are a sum of prefix counts.  With
// C_{P-1} = T3 (the trailing-three table) and C_k[p] = sum_{x >= 0}
// C_{k+1}[p - x h_k] (the trailing tables carried up to level k: the
// factorizations of p over levels k..D-1), the rows before the position with
// prefix (a_0..a_{P-2}), run index b = a_{P-1} and residuals p_0 = n,
// p_{k+1} = p_k - a_k h_k number
//   F = sum_{k <= P-1} (C_k[p_k] - C_k[p_k - a_k h_k]),
// each term the factorizations whose level-k coordinate is below a_k.  Every
// block builds W (leaf counts, for unranking) and C in shared memory (when
// they fit), then its threads unrank slice starts (as k_plan) and write
// slice_off[s] = F(start of s) directly; the total is C_0[n].  The grid also
// writes the pair tables the write walk reads.
__global__ void __launch_bounds__(1024) k_plan_offsets(const __grid_constant__ QueryConst q,
                                                       Scratch sc, uint64_t S_req, int auto_s,
                                                       uint64_t min_leaves, uint64_t* dev_count)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ uint64_t part64[1024];
    __shared__ int32_t part32[1024];
    __shared__ int32_t hs[FS_MAX_D];
    __shared__ Div32 dvh[FS_MAX_D];
    __shared__ uint64_t sS, sL;
    __shared__ SliceSplit ssp;
    const int tid = threadIdx.x;
    const int len = q.n + 1;
    const int P = q.P;
    uint64_t* Ws = (uint64_t*)dyn;               // (P-1) x (n+1) leaf counts
    uint64_t* C = Ws + (size_t)q.nw * len;       // P x (n+1) prefix counts
    if (tid < FS_MAX_D) {
        hs[tid] = q.h[tid];
        dvh[tid] = q.dv_h[tid];
    }
    if (q.tab_xy)  // the write walk's pair tables, spread over the grid
        pair_tables_fill(q, nullptr, sc.X0, sc.YD, blockIdx.x * blockDim.x + tid,
                         gridDim.x * blockDim.x);
    trailing_tables_block(q, 3, C + (size_t)(P - 1) * len, nullptr, nullptr, part64, part32);
    // W_k and C_k are strided prefix sums of W_{k+1} and C_{k+1} with the same
    // stride h_k: one pass for both where the chains are short
    for (int k = P - 2; k >= 0; k--) {
        const uint64_t* in = (k == P - 2) ? nullptr : Ws + (size_t)(k + 1) * len;
        const uint64_t* cin = C + (size_t)(k + 1) * len;
        const int h = q.h[k];
        if (h < len && strided_by_warps(len, h)) {
            warp_chains_scan2([&](int p) { return sps_in(in, p, q.dv_in); }, Ws + (size_t)k * len,
                              [&](int p) { return cin[p]; }, C + (size_t)k * len, len, h);
        } else {
            block_strided_prefix_sum(in, q.dv_in, Ws + (size_t)k * len, len, h, part64);
            block_strided_prefix_sum(cin, q.dv_in, C + (size_t)k * len, len, h, part64);
        }
    }
    if (tid == 0) {
        const uint64_t L = total_leaves(q, Ws);
        uint64_t S = S_req;
        if (auto_s) {
            uint64_t want = (L + min_leaves - 1) / min_leaves;
            if (want < 1) want = 1;
            if (want < S) S = want;
        }
        ssp = make_split(L, S, auto_s);
        sS = S;
        sL = L;
        if (blockIdx.x == 0) {
            sc.ctr[CTR_SEFF] = S;
            sc.ctr[CTR_L] = L;
            record_split(sc.ctr, ssp);
            const uint64_t total = C[q.n];  // C_0[n] = |Z|
            sc.ctr[CTR_TOTAL] = total;
            sc.slice_off[S] = total;
            if (dev_count) *dev_count = total;
        }
    }
    __syncthreads();
    const uint64_t S = sS, L = sL;
    const SliceSplit split = ssp;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t* Clast = C + (size_t)(P - 1) * len;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + tid; s < S; s += nt) {
        int32_t* st = sc.starts + s * START_W;
        const uint64_t k0 = split.start(s);
        if (k0 >= L) {  // empty slice: starts at the end
            st[START_W - 1] = -1;
            sc.slice_off[s] = C[q.n];
            continue;
        }
        // level k < P-1 with residual p before it and coordinate a contributes
        // C_k[p] - C_k[p - a h_k]; level P-1 (index b in the run with residual pr)
        // C_{P-1}[pr] - C_{P-1}[pr - b h_{P-1}]
        uint64_t f = 0;
        int32_t pr;
        const int32_t b = thread_unrank(q, hs, dvh, Ws, k0, pr, [&](int k, int32_t p, int32_t a) {
            st[k] = a;
            const uint64_t* Ck = C + (size_t)k * len;
            f += Ck[p] - Ck[p - a * hs[k]];
        });
        st[START_W - 1] = b;
        sc.slice_off[s] = f + Clast[pr] - Clast[pr - b * hs[P - 1]];
    }
}

size_t plan_runs_smem_bytes(const QueryConst& q)
{
    return ((size_t)q.nw + (size_t)q.P) * (size_t)(q.n + 1) * 8;
}

cudaError_t launch_plan_runs(const QueryConst& q, const Scratch& sc, uint64_t S_req, int auto_s,
                             uint64_t min_leaves, uint64_t* dev_count, cudaStream_t st)
{
    const size_t smem = plan_runs_smem_bytes(q);
    cudaError_t e = smem_optin((const void*)k_plan_offsets, (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = sm_count_cached(&sms);
    if (e != cudaSuccess) return e;
    const uint64_t need = (S_req + 1023) / 1024;  // one slice per thread
    const unsigned blocks = (unsigned)(need < (uint64_t)sms ? need : (uint64_t)sms);
    k_plan_offsets<<<blocks, 1024, smem, st>>>(q, sc, S_req, auto_s, min_leaves, dev_count);
    return cudaGetLastError();
}

// The count modes keep a uint32 copy of the table in shared memory up to
// this size; above it the walk reads the uint64 table through L2.  Where the
// lengths fit 16 bits the length range keeps its tables in shared memory too:
// the count table and the packed range in one walk (MODE 1) while both fit,
// else two walks, the count (MODE 0) and the range alone (MODE 2); beyond
// that one walk reading all three tables through L2.
constexpr int TRIPLE_SMEM_MAX = 160 * 1024;

static int triple_smem(const QueryConst& q3, Op op)
{
    const long long b = ((long long)q3.n + 1) * 4;
    if (b > TRIPLE_SMEM_MAX) return 0;
    if (op != OP_LEN) return (int)b;
    if (q3.maxlen > 0xfffe) return 0;
    return 2 * b <= TRIPLE_SMEM_MAX ? (int)(2 * b) : (int)b;
}

// The length range in two walks (count, then range) rather than one.
static bool triple_len_split(const QueryConst& q3)
{
    const int smem = triple_smem(q3, OP_LEN);
    return smem && (long long)smem < 2 * ((long long)q3.n + 1) * 4;
}

int triple_walk_kernels(const QueryConst& q3, Op op)
{
    return op == OP_LEN && triple_len_split(q3) ? 2 : 1;
}

int triple_threads(const QueryConst& q3, Op op)
{
    return triple_smem(q3, op) > 48 * 1024 ? 1024 : 256;  // big table: one wide block per SM
}

cudaError_t triple_occupancy(const QueryConst& q3, Op op, int threads, int* nb)
{
    const int smem = triple_smem(q3, op);
    if (smem) return occupancy_cached((const void*)k_triple_walk<0, false, true>, threads, smem, nb);
    return occupancy_cached((const void*)k_triple_walk<1, false, false>, threads, 0, nb);
}

// Whether the shared-memory table walk staggers its lanes (walk_slice_packed):
// sibling runs' residuals an even distance apart (bank conflicts) and an odd
// step between a run's leaves.
static bool triple_staggers(const QueryConst& q3)
{
    if (q3.P < 2) return false;
    const int32_t hsib = q3.h[q3.P - 2], hin = q3.h[q3.P - 1];
    return (hsib & 1) == 0 && (hin & 1) == 1;
}

template <int MODE, bool PER_SLICE, bool STAG>
static cudaError_t launch_triple_smem(const QueryConst& q3, const Scratch& sc, dim3 g, dim3 b,
                                      int smem, int queue, const uint64_t* T3, const int32_t* MN3,
                                      const int32_t* MX3, uint64_t* dev_count, cudaStream_t st)
{
    const cudaError_t e = smem_optin((const void*)k_triple_walk<MODE, PER_SLICE, true, STAG>, smem);
    if (e == cudaSuccess)
        k_triple_walk<MODE, PER_SLICE, true, STAG><<<g, b, smem, st>>>(q3, sc, queue, T3, MN3, MX3,
                                                                      dev_count);
    return e;
}

cudaError_t launch_triple(const QueryConst& q3, const Scratch& sc, Op op, const LaunchCfg& lc,
                          int queue, const uint64_t* T3, const int32_t* MN3, const int32_t* MX3,
                          uint64_t* dev_count, cudaStream_t st)
{
    const dim3 g(lc.blocks), b(lc.threads);
    const int smem = triple_smem(q3, op);
    const bool stag = triple_staggers(q3);
    cudaError_t e = cudaSuccess;
    switch (op) {
    case OP_COUNT:
        if (smem) {
            e = stag ? launch_triple_smem<0, false, true>(q3, sc, g, b, smem, queue, T3, nullptr, nullptr, dev_count, st)
                     : launch_triple_smem<0, false, false>(q3, sc, g, b, smem, queue, T3, nullptr, nullptr, dev_count, st);
        } else {
            k_triple_walk<0, false, false><<<g, b, 0, st>>>(q3, sc, queue, T3, MN3, MX3, dev_count);
        }
        break;
    case OP_SLICES:
        if (smem) {
            e = stag ? launch_triple_smem<0, true, true>(q3, sc, g, b, smem, queue, T3, nullptr, nullptr, nullptr, st)
                     : launch_triple_smem<0, true, false>(q3, sc, g, b, smem, queue, T3, nullptr, nullptr, nullptr, st);
        } else {
            k_triple_walk<0, true, false><<<g, b, 0, st>>>(q3, sc, queue, T3, MN3, MX3, nullptr);
        }
        break;
    case OP_LEN:
        if (smem && triple_len_split(q3)) {  // the count, then the range (its own slice queue)
            e = stag ? launch_triple_smem<0, false, true>(q3, sc, g, b, smem, queue, T3, nullptr, nullptr, nullptr, st)
                     : launch_triple_smem<0, false, false>(q3, sc, g, b, smem, queue, T3, nullptr, nullptr, nullptr, st);
            if (e == cudaSuccess)
                e = stag ? launch_triple_smem<2, false, true>(q3, sc, g, b, smem, CTR_QUEUE2, T3, MN3, MX3, nullptr, st)
                         : launch_triple_smem<2, false, false>(q3, sc, g, b, smem, CTR_QUEUE2, T3, MN3, MX3, nullptr, st);
        } else if (smem) {
            e = stag ? launch_triple_smem<1, false, true>(q3, sc, g, b, smem, queue, T3, MN3, MX3, nullptr, st)
                     : launch_triple_smem<1, false, false>(q3, sc, g, b, smem, queue, T3, MN3, MX3, nullptr, st);
        } else {
            k_triple_walk<1, false, false><<<g, b, 0, st>>>(q3, sc, queue, T3, MN3, MX3, nullptr);
        }
        break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ===========================================================================
// launchers
// ===========================================================================
static bool tab_for(const QueryConst& q, Op op)
{
    return (op == OP_COUNT || op == OP_SLICES) ? q.tab_e != 0 : q.tab_xy != 0;
}

// The length walk keeps one 32-bit difference array per warp when the pair
// tables are in use, the lengths step (delta != 0), and the arrays of a block
// fit in HIST_WARP_SMEM_MAX; otherwise one 64-bit array per block (or the
// global one) with the in-walk count, min and max (k_pair_len).
constexpr int HIST_WARP_SMEM_MAX = 64 * 1024;
static bool hist_per_warp(const QueryConst& q, int threads)
{
    return q.tab_xy && q.delta != 0 && hist_smem_bytes(q, threads) <= HIST_WARP_SMEM_MAX;
}

int pair_smem_bytes(const QueryConst& q, Op op, int threads, int elem_bytes)
{
    const bool tab = tab_for(q, op);
    switch (op) {
    case OP_COUNT:
    case OP_SLICES:
        return tab ? (int)(((q.lcm + 31) & ~31u) * 4) : 0;
    case OP_LEN: {
        if (hist_per_warp(q, threads)) return hist_smem_bytes(q, threads);
        int b = tab ? (int)q.lcm * 8 : 0;
        if (q.dbins <= 4096) b += q.dbins * 8;
        return b;
    }
    case OP_ANY:
        return tab ? (int)q.lcm * 8 : 0;
    case OP_ENUM:
        return pair_enum_smem_bytes(q, threads, elem_bytes);
    }
    return 0;
}

template <class K>
static cudaError_t occ(K kern, int threads, int smem, int* nb)
{
    return occupancy_cached((const void*)kern, threads, smem, nb);
}

template <typename... KArgs, typename... Args>
static cudaError_t go(void (*kern)(KArgs...), dim3 g, dim3 b, int smem, cudaStream_t st,
                      Args... args)
{
    cudaError_t e = smem_optin((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<g, b, smem, st>>>(args...);
    return cudaGetLastError();
}

// The count walk's instance for q: table path or not, 32-bit group sums or
// not, the quotient by lcm as one multiply-high or not.
using CountKernel = void (*)(QueryConst, Scratch, int, uint64_t*);
template <bool PER_SLICE>
static CountKernel count_kernel(const QueryConst& q, bool tab)
{
    if (!tab) return k_pair_count<false, PER_SLICE, false>;
    if (!q.acc32) return k_pair_count<true, PER_SLICE, false>;
    return q.fdiv ? k_pair_count<true, PER_SLICE, true, true> : k_pair_count<true, PER_SLICE, true>;
}

cudaError_t pair_occupancy(const QueryConst& q, Op op, int threads, int elem_bytes, int* nb)
{
    const int smem = pair_smem_bytes(q, op, threads, elem_bytes);
    const bool tab = tab_for(q, op);
    switch (op) {
    case OP_COUNT:
        return occ(count_kernel<false>(q, tab), threads, smem, nb);
    case OP_SLICES:
        return occ(count_kernel<true>(q, tab), threads, smem, nb);
    case OP_LEN:
        if (hist_per_warp(q, threads)) return occ(q.fdiv ? k_pair_hist<true> : k_pair_hist<false>, threads, smem, nb);
        if (q.dbins <= 4096)
            return tab ? occ(k_pair_len<true, true>, threads, smem, nb)
                       : occ(k_pair_len<false, true>, threads, smem, nb);
        return tab ? occ(k_pair_len<true, false>, threads, smem, nb)
                   : occ(k_pair_len<false, false>, threads, smem, nb);
    case OP_ANY:
        return tab ? occ(k_pair_any<true>, threads, smem, nb)
                   : occ(k_pair_any<false>, threads, smem, nb);
    case OP_ENUM:
        return pair_enum_occupancy(q, threads, elem_bytes, nb);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_pair(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                        int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                        int elem_bytes, cudaStream_t st)
{
    const int smem = pair_smem_bytes(q, op, lc.threads, elem_bytes);
    const bool tab = tab_for(q, op);
    const dim3 g(lc.blocks), b(lc.threads);
    switch (op) {
    case OP_COUNT:  // `out`: the device total (nullable)
        return go(count_kernel<false>(q, tab), g, b, smem, st, q, sc, queue, (uint64_t*)out);
    case OP_SLICES:
        return go(count_kernel<true>(q, tab), g, b, smem, st, q, sc, queue, (uint64_t*)nullptr);
    case OP_LEN:
        if (hist_per_warp(q, lc.threads))
            return go(q.fdiv ? k_pair_hist<true> : k_pair_hist<false>, g, b, smem, st, q, sc, queue);
        if (q.dbins <= 4096)
            return tab ? go(k_pair_len<true, true>, g, b, smem, st, q, sc, queue)
                       : go(k_pair_len<false, true>, g, b, smem, st, q, sc, queue);
        return tab ? go(k_pair_len<true, false>, g, b, smem, st, q, sc, queue)
                   : go(k_pair_len<false, false>, g, b, smem, st, q, sc, queue);
    case OP_ANY:
        return tab ? go(k_pair_any<true>, g, b, smem, st, q, sc, queue, *pred)
                   : go(k_pair_any<false>, g, b, smem, st, q, sc, queue, *pred);
    case OP_ENUM:
        return launch_pair_enum(q, sc, lc, queue, out, cap_rows, elem_bytes, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fsi
