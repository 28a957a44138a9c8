// The PAIR method: bounded lexicographic walk over the leaves, with the last
// two coordinates of every leaf resolved in closed form (the congruence step
// of Sec. 3.2.4 taken to its end).  Persistent warps pop slices from a device
// queue (Sec. 4: each worker owns a bounded slice of the lex order), and each
// warp walks 32 leaves per step (walk.cuh).  Consumers (Sec. 2): count, length
// statistics, predicate, save (enumerate).
#include "launch.h"
#include "walk.cuh"

namespace fsi {

struct SmemQ {
    int32_t h[FS_MAX_D];
    int32_t col[FS_MAX_D];
    Div32 dvh[FS_MAX_D];
};

FS_D void load_smemq(const QueryConst& q, SmemQ& sq)
{
    const int t = threadIdx.x;
    if (t < FS_MAX_D) {
        sq.h[t] = q.h[t];
        sq.col[t] = q.col[t];
        sq.dvh[t] = q.dv_h[t];
    }
}

// Pop slices from the queue and walk each one with `cons`.
template <class Cons>
FS_D void run_queue(const QueryConst& q, const SmemQ& sq, const Scratch& sc, uint64_t S, int queue,
                    Cons& cons)
{
    const int lane = threadIdx.x & 31;
    const int32_t hk = lane < q.P - 1 ? sq.h[lane] : 0;
    const uint64_t L = total_leaves(q, sc.W);
    unsigned long long* qc = (unsigned long long*)&sc.ctr[queue];
    for (;;) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(qc, 1ull);
        s = __shfl_sync(FULL, s, 0);
        if (s >= S) break;
        const uint64_t k0 = slice_start(s, L, S), k1 = slice_start(s + 1, L, S);
        cons.slice_begin(q, s);
        bool stop = false;
        if (k1 > k0) stop = walk_slice(q, sq.h, sq.dvh, sc.W, k0, k1 - k0, lane, hk, cons);
        cons.slice_end(q, s);
        if (stop) break;
    }
}

// ===========================================================================
// count
// ===========================================================================
// Sets the device error flag the host checks after a synchronous call.
FS_D void flag_fault(uint64_t* ctr)
{
    if ((threadIdx.x & 31) == 0) atomicOr((unsigned long long*)&ctr[CTR_ERR], 1ull);
}

template <bool TAB, bool PER_SLICE>
struct CountCons {
    const int8_t* E;
    uint64_t* slice_cnt;
    uint64_t acc;    // this lane, current slice
    uint64_t total;  // this lane, all slices
    uint64_t* ctr;
    FS_D void fault() { flag_fault(ctr); }
    FS_D void run_loaded(const QueryConst&, int, const RunPrefix&, int) {}
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
    FS_D bool chunk(const QueryConst& q, int, bool valid, int32_t r, int32_t, int32_t, int)
    {
        if (valid) acc += pair_count<TAB>(q, E, r);
        return false;
    }
};

template <bool TAB, bool PER_SLICE>
__global__ void __launch_bounds__(256) k_pair_count(const __grid_constant__ QueryConst q,
                                                    Scratch sc, uint64_t S, int queue)
{
    __shared__ SmemQ sq;
    __shared__ unsigned long long bsum;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq);
    if (threadIdx.x == 0) bsum = 0;
    int8_t* E = (int8_t*)dyn;
    if (TAB)
        for (uint32_t i = threadIdx.x; i < q.lcm; i += blockDim.x) E[i] = sc.E[i];
    __syncthreads();
    CountCons<TAB, PER_SLICE> cons{E, sc.slice_cnt, 0, 0, sc.ctr};
    run_queue(q, sq, sc, S, queue, cons);
    uint64_t v = warp_sum_u64(cons.total);
    if ((threadIdx.x & 31) == 0) atomicAdd(&bsum, (unsigned long long)v);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&sc.ctr[CTR_COUNT], bsum);
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
    FS_D void fault() { flag_fault(ctr); }
    FS_D void run_loaded(const QueryConst&, int, const RunPrefix&, int) {}
    FS_D void slice_begin(const QueryConst&, uint64_t) {}
    FS_D void slice_end(const QueryConst&, uint64_t) {}
    FS_D bool chunk(const QueryConst& q, int, bool valid, int32_t r, int32_t a, int32_t lp, int)
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
                                                  Scratch sc, uint64_t S, int queue)
{
    __shared__ SmemQ sq;
    __shared__ unsigned long long bsum;
    __shared__ unsigned int bmin, bmax;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq);
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
    run_queue(q, sq, sc, S, queue, cons);
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
    int64_t pw0, pw1;  // weighted prefix sums of the runs in slots 0 / 1
    int poll;
    uint64_t* ctr;
    FS_D void fault() { flag_fault(ctr); }
    FS_D void run_loaded(const QueryConst& q, int slot, const RunPrefix& rp, int lane)
    {
        int64_t v = (lane < q.P - 1) ? pc->w[lane] * (int64_t)rp.a : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (slot == 0) pw0 = v; else pw1 = v;
    }
    FS_D void slice_begin(const QueryConst&, uint64_t) {}
    FS_D void slice_end(const QueryConst&, uint64_t) {}
    FS_D bool chunk(const QueryConst& q, int lane, bool valid, int32_t r, int32_t a, int32_t,
                    int slot)
    {
        bool f = false;
        if (valid) {
            int32_t x0 = 0, y0 = 0;
            uint32_t c = pair_xy<TAB>(q, X0, YD, r, x0, y0);
            if (c > 0) {
                int64_t V0 = (slot ? pw1 : pw0) + pc->w[q.P - 1] * (int64_t)a +
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
__global__ void __launch_bounds__(256) k_pair_any(const __grid_constant__ QueryConst q,
                                                  Scratch sc, uint64_t S, int queue,
                                                  const __grid_constant__ PredConst pred)
{
    __shared__ SmemQ sq;
    __shared__ PredConst spc;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq);
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
    run_queue(q, sq, sc, S, queue, cons);
}

// ===========================================================================
// enumerate (second walk): rows of the slice written at the slice's offset
// ===========================================================================
// Rows are staged per warp in shared memory and written out as 16-byte
// streaming stores.  Within a chunk the rows of lane l's leaf follow those of
// lanes < l (warp scan of the counts), so each slice writes its rows in lex
// order into [off_s, off_s + count_s).
enum { ENUM_STG_BYTES = 6144, ENUM_MAPCAP = 256, ENUM_BIG = 1 << 26 };
enum { ENUM_WARP_BYTES = ENUM_STG_BYTES + 2 * FS_MAX_D * 4 + ENUM_MAPCAP };

template <bool TAB, typename ELEM>
struct EnumCons {
    static constexpr int VEC = 16 / (int)sizeof(ELEM);
    static constexpr int STG = ENUM_STG_BYTES / (int)sizeof(ELEM);
    const int32_t* X0;
    const int32_t* YD;
    const int32_t* col;
    const uint64_t* slice_off;
    ELEM* out;
    uint64_t cap_elems;
    ELEM* stg;
    int32_t* tmpl;   // [2][FS_MAX_D], by walk level
    uint8_t* map;    // row -> lane, ENUM_MAPCAP
    uint64_t row_base;
    int32_t nst;
    int32_t phase;
    int32_t d;
    int32_t piece;   // rows per piece
    uint64_t* ctr;
    FS_D void fault() { flag_fault(ctr); }

    FS_D void run_loaded(const QueryConst& q, int slot, const RunPrefix& rp, int lane)
    {
        if (lane < q.P - 1) tmpl[slot * FS_MAX_D + lane] = rp.a;
        __syncwarp();
    }
    FS_D void slice_begin(const QueryConst&, uint64_t s)
    {
        row_base = slice_off[s];
        nst = 0;
        phase = (int32_t)((row_base * (uint64_t)d) % VEC);
    }
    FS_D void flush()
    {
        const int lane = threadIdx.x & 31;
        if (nst > 0) {
            const uint64_t g0 = row_base * (uint64_t)d;
            const uint64_t N = (uint64_t)nst * (uint64_t)d;
            const uint64_t gend = (g0 + N < cap_elems) ? g0 + N : cap_elems;
            if (g0 < gend) {
                const uint64_t vb = (g0 + VEC - 1) / VEC, ve = gend / VEC;
                if (vb < ve) {
                    const uint64_t head = vb * VEC - g0;
                    for (uint64_t i = lane; i < head; i += 32) out[g0 + i] = stg[phase + i];
                    const uint4* sv = reinterpret_cast<const uint4*>(stg + phase + head);
                    uint4* gv = reinterpret_cast<uint4*>(out) + vb;
                    const uint64_t nv = ve - vb;
                    for (uint64_t j = lane; j < nv; j += 32) __stcs(gv + j, sv[j]);
                    for (uint64_t i = ve * VEC + lane; i < gend; i += 32)
                        out[i] = stg[phase + (i - g0)];
                } else {
                    for (uint64_t i = lane; i < gend - g0; i += 32) out[g0 + i] = stg[phase + i];
                }
            }
        }
        row_base += (uint64_t)nst;
        nst = 0;
        phase = (int32_t)((row_base * (uint64_t)d) % VEC);
        __syncwarp();
    }
    FS_D void slice_end(const QueryConst&, uint64_t) { flush(); }

    // Emit the T rows of one chunk: lane l owns rows [excl, incl).
    FS_D void emit(const QueryConst& q, int lane, uint32_t T, uint32_t excl, uint32_t incl,
                   int32_t x0, int32_t y0, int32_t a, int slot)
    {
        for (uint32_t ps = 0; ps < T; ps += piece) {
            const uint32_t np = min((uint32_t)piece, T - ps);
            if (phase + (nst + (int32_t)np) * d > STG) flush();
            const uint32_t lo = max(excl, ps), hi = min(incl, ps + np);
            for (uint32_t i = lo; i < hi; i++) map[i - ps] = (uint8_t)lane;
            __syncwarp();
            for (uint32_t j = 0; j < np; j += 32) {
                const uint32_t i = j + lane;
                const bool ok = i < np;
                const int src = ok ? map[i] : 0;
                const uint32_t es = __shfl_sync(FULL, excl, src);
                const int32_t xs = __shfl_sync(FULL, x0, src);
                const int32_t ys = __shfl_sync(FULL, y0, src);
                const int32_t as = __shfl_sync(FULL, a, src);
                const int ss = __shfl_sync(FULL, slot, src);
                if (ok) {
                    const int32_t t = (int32_t)(ps + i - es);
                    ELEM* row = stg + phase + (nst + (int32_t)i) * d;
                    const int32_t* tp = tmpl + ss * FS_MAX_D;
                    for (int k = 0; k < q.P - 1; k++) {
                        const int c = col[k];
                        if (c >= 0) row[c] = (ELEM)tp[k];
                    }
                    int c = col[q.P - 1];
                    if (c >= 0) row[c] = (ELEM)as;
                    c = col[q.P];
                    if (c >= 0) row[c] = (ELEM)(xs + t * q.v);
                    c = col[q.P + 1];
                    if (c >= 0) row[c] = (ELEM)(ys - t * q.u);
                }
            }
            nst += (int32_t)np;
            __syncwarp();
        }
    }

    FS_D bool chunk(const QueryConst& q, int lane, bool valid, int32_t r, int32_t a, int32_t,
                    int slot)
    {
        int32_t x0 = 0, y0 = 0;
        uint32_t c = 0;
        if (valid) c = pair_xy<TAB>(q, X0, YD, r, x0, y0);
        if (__any_sync(FULL, c > (uint32_t)ENUM_BIG)) {
            // rare: a leaf with a huge number of rows; one leaf at a time
            for (int src = 0; src < 32; src++) {
                const uint32_t cs = __shfl_sync(FULL, c, src);
                if (cs == 0) continue;
                const bool me = lane == src;
                emit(q, lane, cs, me ? 0u : cs, me ? cs : cs, x0, y0, a, slot);
            }
            return false;
        }
        uint32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t T = __shfl_sync(FULL, incl, 31);
        if (T > 0) emit(q, lane, T, incl - c, incl, x0, y0, a, slot);
        return false;
    }
};

template <bool TAB, typename ELEM>
__global__ void __launch_bounds__(256) k_pair_enum(const __grid_constant__ QueryConst q,
                                                   Scratch sc, uint64_t S, int queue, ELEM* out,
                                                   uint64_t cap_rows)
{
    __shared__ SmemQ sq;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq);
    int32_t* X0 = (int32_t*)dyn;
    int32_t* YD = X0 + (TAB ? q.lcm : 0);
    if (TAB)
        for (uint32_t i = threadIdx.x; i < q.lcm; i += blockDim.x) {
            X0[i] = sc.X0[i];
            YD[i] = sc.YD[i];
        }
    const size_t tab = TAB ? (((size_t)q.lcm * 8 + 15) & ~(size_t)15) : 0;
    unsigned char* wp = dyn + tab + (size_t)(threadIdx.x >> 5) * ENUM_WARP_BYTES;
    __syncthreads();
    EnumCons<TAB, ELEM> cons;
    cons.X0 = X0;
    cons.YD = YD;
    cons.col = sq.col;
    cons.slice_off = sc.slice_off;
    cons.out = out;
    cons.cap_elems = cap_rows * (uint64_t)q.d;
    cons.stg = (ELEM*)wp;
    cons.tmpl = (int32_t*)(wp + ENUM_STG_BYTES);
    cons.map = wp + ENUM_STG_BYTES + 2 * FS_MAX_D * 4;
    cons.row_base = 0;
    cons.nst = 0;
    cons.phase = 0;
    cons.d = q.d;
    int piece = (EnumCons<TAB, ELEM>::STG - EnumCons<TAB, ELEM>::VEC) / q.d;
    cons.piece = piece < ENUM_MAPCAP ? piece : ENUM_MAPCAP;
    cons.ctr = sc.ctr;
    run_queue(q, sq, sc, S, queue, cons);
}

// ===========================================================================
// launchers
// ===========================================================================
static bool tab_for(const QueryConst& q, Op op)
{
    return (op == OP_COUNT || op == OP_SLICES) ? q.tab_e != 0 : q.tab_xy != 0;
}

int pair_smem_bytes(const QueryConst& q, Op op, int threads, int elem_bytes)
{
    const bool tab = tab_for(q, op);
    switch (op) {
    case OP_COUNT:
    case OP_SLICES:
        return tab ? (int)q.lcm : 0;
    case OP_LEN: {
        int b = tab ? (int)q.lcm * 8 : 0;
        if (q.dbins <= 4096) b += q.dbins * 8;
        return b;
    }
    case OP_ANY:
        return tab ? (int)q.lcm * 8 : 0;
    case OP_ENUM: {
        int b = tab ? (((int)q.lcm * 8 + 15) & ~15) : 0;
        return b + (threads / 32) * ENUM_WARP_BYTES;
    }
    }
    (void)elem_bytes;
    return 0;
}

template <class K>
static cudaError_t occ(K kern, int threads, int smem, int* nb)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, threads, smem);
}

template <class K>
static cudaError_t prep(K kern, int smem)
{
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return cudaSuccess;
}

cudaError_t pair_occupancy(const QueryConst& q, Op op, int threads, int elem_bytes, int* nb)
{
    const int smem = pair_smem_bytes(q, op, threads, elem_bytes);
    const bool tab = tab_for(q, op);
    switch (op) {
    case OP_COUNT:
        return tab ? occ(k_pair_count<true, false>, threads, smem, nb)
                   : occ(k_pair_count<false, false>, threads, smem, nb);
    case OP_SLICES:
        return tab ? occ(k_pair_count<true, true>, threads, smem, nb)
                   : occ(k_pair_count<false, true>, threads, smem, nb);
    case OP_LEN:
        if (q.dbins <= 4096)
            return tab ? occ(k_pair_len<true, true>, threads, smem, nb)
                       : occ(k_pair_len<false, true>, threads, smem, nb);
        return tab ? occ(k_pair_len<true, false>, threads, smem, nb)
                   : occ(k_pair_len<false, false>, threads, smem, nb);
    case OP_ANY:
        return tab ? occ(k_pair_any<true>, threads, smem, nb)
                   : occ(k_pair_any<false>, threads, smem, nb);
    case OP_ENUM:
        if (elem_bytes == 2)
            return tab ? occ(k_pair_enum<true, int16_t>, threads, smem, nb)
                       : occ(k_pair_enum<false, int16_t>, threads, smem, nb);
        return tab ? occ(k_pair_enum<true, int32_t>, threads, smem, nb)
                   : occ(k_pair_enum<false, int32_t>, threads, smem, nb);
    }
    return cudaErrorInvalidValue;
}

template <typename... KArgs, typename... Args>
static cudaError_t go(void (*kern)(KArgs...), dim3 g, dim3 b, int smem, cudaStream_t st,
                      Args... args)
{
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<g, b, smem, st>>>(args...);
    return cudaGetLastError();
}

cudaError_t launch_pair(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                        int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                        int elem_bytes, cudaStream_t st)
{
    const int smem = pair_smem_bytes(q, op, lc.threads, elem_bytes);
    const bool tab = tab_for(q, op);
    const dim3 g(lc.blocks), b(lc.threads);
    const uint64_t S = lc.S;
    switch (op) {
    case OP_COUNT:
        return tab ? go(k_pair_count<true, false>, g, b, smem, st, q, sc, S, queue)
                   : go(k_pair_count<false, false>, g, b, smem, st, q, sc, S, queue);
    case OP_SLICES:
        return tab ? go(k_pair_count<true, true>, g, b, smem, st, q, sc, S, queue)
                   : go(k_pair_count<false, true>, g, b, smem, st, q, sc, S, queue);
    case OP_LEN:
        if (q.dbins <= 4096)
            return tab ? go(k_pair_len<true, true>, g, b, smem, st, q, sc, S, queue)
                       : go(k_pair_len<false, true>, g, b, smem, st, q, sc, S, queue);
        return tab ? go(k_pair_len<true, false>, g, b, smem, st, q, sc, S, queue)
                   : go(k_pair_len<false, false>, g, b, smem, st, q, sc, S, queue);
    case OP_ANY:
        return tab ? go(k_pair_any<true>, g, b, smem, st, q, sc, S, queue, *pred)
                   : go(k_pair_any<false>, g, b, smem, st, q, sc, S, queue, *pred);
    case OP_ENUM:
        if (elem_bytes == 2)
            return tab ? go(k_pair_enum<true, int16_t>, g, b, smem, st, q, sc, S, queue,
                            (int16_t*)out, cap_rows)
                       : go(k_pair_enum<false, int16_t>, g, b, smem, st, q, sc, S, queue,
                            (int16_t*)out, cap_rows);
        return tab ? go(k_pair_enum<true, int32_t>, g, b, smem, st, q, sc, S, queue,
                        (int32_t*)out, cap_rows)
                   : go(k_pair_enum<false, int32_t>, g, b, smem, st, q, sc, S, queue,
                        (int32_t*)out, cap_rows);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fsi
