// The PLAIN method: the paper's successor (nextCandidate, Sec. 3.2.2) with no
// shortcut, one bounded stream per GPU thread with the whole state in registers
// (Sec. 3.1.2, Sec. 5).  A thread pops a slice [lo, hi) from the device queue,
// starts at hi (or at the first candidate of Sec. 3.2.1 for the last slice),
// and steps nextCandidate until the candidate drops below lo, consuming the
// candidates whose wasValid is set (Sec. 3.3: the caller filters).
#include "launch.h"
#include "walk.cuh"

namespace fsi {

struct SmemQP {
    int32_t h[FS_MAX_D];
    int32_t col[FS_MAX_D];
    Div32 dvh[FS_MAX_D];
};

// Slice s's start as a full vector (leaf, 0, 0) from the planner's table.
template <int MAXD>
FS_D void load_start_thread(const QueryConst& q, const int32_t* starts, uint64_t s,
                            int32_t (&v)[MAXD])
{
    const int32_t* st = starts + s * START_W;
#pragma unroll
    for (int k = 0; k < MAXD; k++) v[k] = (k < q.P - 1) ? st[k] : 0;
#pragma unroll
    for (int k = 0; k < MAXD; k++)
        if (k == q.P - 1) v[k] = st[START_W - 1];
}

// The successor of a candidate in the lex-decreasing stream (nextCandidate,
// Sec. 3.2.2): the pivot is the last nonzero coordinate before the final one;
// it drops by one, the coordinates right of it are cleared, and the one just
// right of it takes the least value that brings phi up to at least n (the
// ceiling of the residual over its generator; the residual is at least 1, as
// the pivot's prefix was reached from below n).  The new candidate is a
// factorization exactly when that division is exact, and by Thm 3.2 none is
// skipped.  Returns false when there is no pivot or the candidate falls below
// the slice's lower bound `lo`; otherwise sets `valid` (wasValid).
template <int MAXD>
FS_D bool next_candidate(const QueryConst& q, const SmemQP& sq, int32_t (&a)[MAXD],
                         const int32_t (&lo)[MAXD], bool& valid)
{
    const int D = q.D;
    int piv = -1;
#pragma unroll
    for (int k = 0; k < MAXD - 1; k++)
        if (k < D - 1 && a[k] > 0) piv = k;
    if (piv < 0) return false;
    // lower the pivot and clear the rest: right of the pivot only the final
    // coordinate can be nonzero
#pragma unroll
    for (int k = 0; k < MAXD; k++) {
        if (k == D - 1) a[k] = 0;
        if (k == piv) a[k] -= 1;
    }
    int64_t phi = 0;
#pragma unroll
    for (int k = 0; k < MAXD; k++)
        if (k < D) phi += (int64_t)a[k] * sq.h[k];
    const int32_t rest = q.n - (int32_t)phi;
    const int32_t hn = sq.h[piv + 1];
    int32_t m = (int32_t)div32((uint32_t)rest, sq.dvh[piv + 1]);
    valid = m * hn == rest;
    if (!valid) m += 1;
#pragma unroll
    for (int k = 0; k < MAXD; k++)
        if (k == piv + 1) a[k] = m;
    // lex comparison with the slice's lower bound
    int cmp = 0;
#pragma unroll
    for (int k = 0; k < MAXD; k++)
        if (cmp == 0 && k < D) cmp = (a[k] < lo[k]) ? -1 : (a[k] > lo[k] ? 1 : 0);
    return cmp >= 0;
}

// Walk one slice; cons.emit(a) is called for every valid candidate in the
// paper's (lex-decreasing) order.  Returns true if the consumer stopped.
template <int MAXD, class Cons>
FS_D bool plain_slice(const QueryConst& q, const SmemQP& sq, const int32_t* starts, uint64_t s,
                      uint64_t k1, uint64_t L, Cons& cons)
{
    int32_t lo[MAXD], a[MAXD];
    load_start_thread<MAXD>(q, starts, s, lo);
    bool valid = false;
    if (k1 == L) {
        // the first candidate (x, 0, .., 0), x = ceil(n / g_1)  (Sec. 3.2.1)
#pragma unroll
        for (int k = 0; k < MAXD; k++) a[k] = 0;
        const int32_t h0 = sq.h[0];
        int32_t x = (int32_t)div32((uint32_t)q.n, sq.dvh[0]);
        if (x * h0 != q.n) x += 1;
        a[0] = x;
        valid = (int64_t)x * h0 == q.n;
        if (valid && cons.emit(q, sq, a)) return true;
    } else {
        // start at the next slice's lower bound (not part of this slice)
        load_start_thread<MAXD>(q, starts, s + 1, a);
    }
    while (next_candidate<MAXD>(q, sq, a, lo, valid)) {
        if (valid && cons.emit(q, sq, a)) return true;
        if (cons.poll()) return true;
    }
    return false;
}

template <int MAXD, class Cons>
FS_D void plain_queue(const QueryConst& q, const SmemQP& sq, const Scratch& sc, int queue,
                      Cons& cons)
{
    const uint64_t S = sc.ctr[CTR_SEFF];
    const uint64_t L = sc.ctr[CTR_L];
    const SliceSplit split = planned_split(sc.ctr);
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long* qc = (unsigned long long*)&sc.ctr[queue];
    // thread t takes slice t first, then pops T, T+1, ... from the queue
    unsigned long long s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (;; s = atomicAdd(qc, 1ull) + T) {
        if (s >= S) break;
        const uint64_t k0 = split.start(s), k1 = split.start(s + 1);
        cons.slice_begin(sc, s);
        bool stop = false;
        if (k1 > k0) stop = plain_slice<MAXD>(q, sq, sc.starts, s, k1, L, cons);
        cons.slice_end(sc, s);
        if (stop) break;
    }
}

FS_D void load_sqp(const QueryConst& q, SmemQP& sq)
{
    const int t = threadIdx.x;
    if (t < FS_MAX_D) {
        sq.h[t] = q.h[t];
        sq.col[t] = q.col[t];
        sq.dvh[t] = q.dv_h[t];
    }
}

// ---------------------------------------------------------------------------
// consumers
// ---------------------------------------------------------------------------
struct PCount {
    uint64_t acc, total;
    bool per_slice;
    template <int MAXD>
    FS_D bool emit(const QueryConst&, const SmemQP&, const int32_t (&)[MAXD])
    {
        acc++;
        return false;
    }
    FS_D bool poll() { return false; }
    FS_D void slice_begin(const Scratch&, uint64_t) { acc = 0; }
    FS_D void slice_end(const Scratch& sc, uint64_t s)
    {
        if (per_slice) sc.slice_cnt[s] = acc;
        total += acc;
    }
};

struct PLen {
    unsigned long long* H;  // histogram (shared or global)
    uint64_t cnt;
    uint32_t mn, mx;
    template <int MAXD>
    FS_D bool emit(const QueryConst& q, const SmemQP&, const int32_t (&a)[MAXD])
    {
        int32_t l = 0;
#pragma unroll
        for (int k = 0; k < MAXD; k++)
            if (k < q.D) l += a[k];
        cnt++;
        mn = min(mn, (uint32_t)l);
        mx = max(mx, (uint32_t)l);
        atomicAdd(&H[l], 1ull);
        return false;
    }
    FS_D bool poll() { return false; }
    FS_D void slice_begin(const Scratch&, uint64_t) {}
    FS_D void slice_end(const Scratch&, uint64_t) {}
};

struct PAny {
    const PredConst* pc;
    unsigned long long* flag;
    uint32_t since;
    template <int MAXD>
    FS_D bool emit(const QueryConst& q, const SmemQP&, const int32_t (&a)[MAXD])
    {
        int64_t v = 0;
#pragma unroll
        for (int k = 0; k < MAXD; k++)
            if (k < q.D) v += pc->w[k] * (int64_t)a[k];
        bool f;
        if (pc->modulus > 0) {
            int64_t M = pc->modulus;
            int64_t vm = v % M;
            if (vm < 0) vm += M;
            int64_t cm = pc->c % M;
            if (cm < 0) cm += M;
            f = vm == cm;
        } else if (pc->op == 0) {
            f = v == pc->c;
        } else if (pc->op == 1) {
            f = v <= pc->c;
        } else {
            f = v >= pc->c;
        }
        if (f) atomicExch(flag, 1ull);
        return f;
    }
    FS_D bool poll()
    {
        if (++since < 1024) return false;
        since = 0;
        return *(volatile unsigned long long*)flag != 0;
    }
    FS_D void slice_begin(const Scratch&, uint64_t) {}
    FS_D void slice_end(const Scratch&, uint64_t) {}
};

template <typename ELEM>
struct PEnum {
    ELEM* out;
    uint64_t cap_rows;
    uint64_t row;   // next row index (written downwards)
    template <int MAXD>
    FS_D bool emit(const QueryConst& q, const SmemQP& sq, const int32_t (&a)[MAXD])
    {
        row--;
        if (row < cap_rows) {
            ELEM* o = out + row * (uint64_t)q.d;
#pragma unroll
            for (int k = 0; k < MAXD; k++)
                if (k < q.D && sq.col[k] >= 0) o[sq.col[k]] = (ELEM)a[k];
        }
        return false;
    }
    FS_D bool poll() { return false; }
    // the stream is lex-decreasing; rows go from the slice's end downwards so
    // that the buffer is lex-ascending, as with the PAIR method
    FS_D void slice_begin(const Scratch& sc, uint64_t s) { row = slice_row0(sc, s + 1); }
    FS_D void slice_end(const Scratch&, uint64_t) {}
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <int MAXD, bool PER_SLICE>
__global__ void __launch_bounds__(128) k_plain_count(const __grid_constant__ QueryConst q,
                                                     Scratch sc, int queue)
{
    __shared__ SmemQP sq;
    __shared__ unsigned long long bsum;
    load_sqp(q, sq);
    if (threadIdx.x == 0) bsum = 0;
    __syncthreads();
    PCount c{0, 0, PER_SLICE};
    plain_queue<MAXD>(q, sq, sc, queue, c);
    uint64_t v = warp_sum_u64(c.total);
    if ((threadIdx.x & 31) == 0) atomicAdd(&bsum, (unsigned long long)v);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&sc.ctr[CTR_COUNT], bsum);
}

template <int MAXD, bool SMEMH>
__global__ void __launch_bounds__(128) k_plain_len(const __grid_constant__ QueryConst q,
                                                   Scratch sc, int queue)
{
    __shared__ SmemQP sq;
    __shared__ unsigned long long bsum;
    __shared__ unsigned int bmin, bmax;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_sqp(q, sq);
    if (threadIdx.x == 0) {
        bsum = 0;
        bmin = 0xffffffffu;
        bmax = 0;
    }
    const int bins = q.maxlen + 1;
    unsigned long long* H = (unsigned long long*)sc.D;
    if (SMEMH) {
        H = (unsigned long long*)dyn;
        for (int i = threadIdx.x; i < bins; i += blockDim.x) H[i] = 0;
    }
    __syncthreads();
    PLen c{H, 0, 0xffffffffu, 0};
    plain_queue<MAXD>(q, sq, sc, queue, c);
    uint64_t v = warp_sum_u64(c.cnt);
    uint32_t mn = c.mn, mx = c.mx;
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
    if (SMEMH)
        for (int i = threadIdx.x; i < bins; i += blockDim.x)
            if (H[i]) atomicAdd((unsigned long long*)&sc.D[i], H[i]);
}

template <int MAXD>
__global__ void __launch_bounds__(128) k_plain_any(const __grid_constant__ QueryConst q,
                                                   Scratch sc, int queue,
                                                   const __grid_constant__ PredConst pred)
{
    __shared__ SmemQP sq;
    __shared__ PredConst spc;
    load_sqp(q, sq);
    if (threadIdx.x == 0) spc = pred;
    __syncthreads();
    PAny c{&spc, (unsigned long long*)&sc.ctr[CTR_FOUND], 0};
    plain_queue<MAXD>(q, sq, sc, queue, c);
}

template <int MAXD, typename ELEM>
__global__ void __launch_bounds__(128) k_plain_enum(const __grid_constant__ QueryConst q,
                                                    Scratch sc, int queue, ELEM* out,
                                                    uint64_t cap_rows)
{
    __shared__ SmemQP sq;
    load_sqp(q, sq);
    __syncthreads();
    PEnum<ELEM> c{out, cap_rows, 0};
    plain_queue<MAXD>(q, sq, sc, queue, c);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename... KArgs, typename... Args>
static cudaError_t go(void (*kern)(KArgs...), dim3 g, dim3 b, int smem, cudaStream_t st,
                      Args... args)
{
    cudaError_t e = smem_optin((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<g, b, smem, st>>>(args...);
    return cudaGetLastError();
}

static int plain_smem(const QueryConst& q, Op op)
{
    if (op == OP_LEN && q.maxlen + 1 <= 4096) return (q.maxlen + 1) * 8;
    return 0;
}

template <int MAXD>
static cudaError_t launch_plain_t(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                                  int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                                  int elem_bytes, cudaStream_t st)
{
    const dim3 g(lc.blocks), b(lc.threads);
    const int smem = plain_smem(q, op);
        switch (op) {
    case OP_COUNT:
        return go(k_plain_count<MAXD, false>, g, b, 0, st, q, sc, queue);
    case OP_SLICES:
        return go(k_plain_count<MAXD, true>, g, b, 0, st, q, sc, queue);
    case OP_LEN:
        return smem ? go(k_plain_len<MAXD, true>, g, b, smem, st, q, sc, queue)
                    : go(k_plain_len<MAXD, false>, g, b, 0, st, q, sc, queue);
    case OP_ANY:
        return go(k_plain_any<MAXD>, g, b, 0, st, q, sc, queue, *pred);
    case OP_ENUM:
        if (elem_bytes == 2)
            return go(k_plain_enum<MAXD, int16_t>, g, b, 0, st, q, sc, queue, (int16_t*)out,
                      cap_rows);
        return go(k_plain_enum<MAXD, int32_t>, g, b, 0, st, q, sc, queue, (int32_t*)out,
                  cap_rows);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_plain(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                         int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                         int elem_bytes, cudaStream_t st)
{
    if (q.D <= 4) return launch_plain_t<4>(q, sc, op, lc, queue, pred, out, cap_rows, elem_bytes, st);
    if (q.D <= 8) return launch_plain_t<8>(q, sc, op, lc, queue, pred, out, cap_rows, elem_bytes, st);
    return launch_plain_t<16>(q, sc, op, lc, queue, pred, out, cap_rows, elem_bytes, st);
}

cudaError_t plain_occupancy(const QueryConst& q, Op op, int threads, int* nb)
{
    const int smem = plain_smem(q, op);
    if (q.D <= 4) return occupancy_cached((const void*)k_plain_count<4, true>, threads, smem, nb);
    if (q.D <= 8) return occupancy_cached((const void*)k_plain_count<8, true>, threads, smem, nb);
    return occupancy_cached((const void*)k_plain_count<16, true>, threads, smem, nb);
}

}  // namespace fsi
