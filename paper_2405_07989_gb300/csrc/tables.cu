// Per-query precompute and finalisation kernels.
//
//  k_precompute   one block per table: the pair tables E / X0 / YD indexed by
//                 r mod lcm(A, B) (closed form of the congruence step, Sec.
//                 3.2.4), the exact leaf counts W_k[p] that the slice planner
//                 unranks (balanced division of labour, Sec. 4.1 and 6.2), the
//                 trailing-k tables (Sec. 6.1)
//  k_plan(_smem)  the slice planner: slice count and each slice's start state
//  k_scan_slices  exclusive scan of per-slice counts -> output offsets
//  k_len_finalize histogram from the strided difference array
//  k_copy_u64     a device counter to the caller's memory
#include "launch.h"
#include "walk.cuh"

namespace fsi {

// All per-query tables of a call in one launch, one role per block (the roles
// are independent): the walk query's leaf counts W, its pair tables, and the
// trailing-k tables of the original query.
//
// Leaf counts: W_k[p] = #{(a_k..a_{P-1}) >= 0 : sum_{i >= k} a_i h_i <= p} for
// k = 0..P-2, p = 0..n.  W_k = W_{k+1} / (1 - x^{h_k}) as series, i.e. a strided
// prefix sum; W_{P-1}[p] = floor(p / h_{P-1}) + 1 in closed form.
// Pair tables: for w in [0, lcm), whether w = x A + y B is solvable "within one
// period" and where the solutions of r = q lcm + w start (see pair_count).
// Trailing-k tables (Sec. 6.1: keep the factorizations of every small
// residual over the trailing generators, here their count and length range).
// For k = 3, with h = h_{P-1} and the pair (A, B) of q, for p = 0..n:
//   T[p]  = #{(a, x, y) >= 0 : a h + x A + y B = p} = sum_{a >= 0} c2(p - a h)
//   MN[p] = min of a + x + y over those solutions (TRIPLE_NONE if none)
//   MX[p] = max of a + x + y (-TRIPLE_NONE if none)
// c2 and the pair's length range come from the pair's closed form (its lengths
// run l0 + t delta); the sums over a are strided scans: a running sum, and a
// running min / max of (bound - floor(p/h)) plus floor(p/h).  k = 4 adds level
// P-2 the same way: T4[p] = sum_{b >= 0} T3[p - b h_{P-2}], and so on for the
// length range.  One block per table (the count, the minimum, the maximum).
struct PrecompArgs {
    QueryConst qw;  // the query the walk runs over
    QueryConst qt;  // the query whose trailing tables are built (trail_k > 0)
    uint64_t* W;
    int8_t* E;
    int32_t* X0;
    int32_t* YD;
    uint64_t* T;
    int32_t* MN;
    int32_t* MX;
    uint64_t* tmax;  // the trailing table's largest entry (ctr[CTR_TMAX])
    int32_t trail_k;
    int32_t nroles;
    int32_t role[6];
};
enum { ROLE_WEIGHTS = 0, ROLE_PAIRTAB = 1, ROLE_TRAIL = 2, ROLE_TRAIL_MN = 3, ROLE_TRAIL_MX = 4 };

__global__ void __launch_bounds__(1024) k_precompute(const __grid_constant__ PrecompArgs a)
{
    __shared__ uint64_t part64[1024];
    __shared__ int32_t part32[1024];
    switch (a.role[blockIdx.x]) {
    case ROLE_WEIGHTS: {
        const QueryConst& q = a.qw;
        const int len = q.n + 1;
        for (int k = q.P - 2; k >= 0; k--) {
            const uint64_t* in = (k == q.P - 2) ? nullptr : a.W + (size_t)(k + 1) * len;
            block_strided_prefix_sum(in, q.dv_in, a.W + (size_t)k * len, len, q.h[k], part64);
        }
        break;
    }
    case ROLE_PAIRTAB:
        pair_tables_fill(a.qw, a.E, a.X0, a.YD, threadIdx.x, blockDim.x);
        break;
    case ROLE_TRAIL:
        trailing_tables_block(a.qt, a.trail_k, a.T, nullptr, nullptr, part64, part32, a.tmax);
        break;
    case ROLE_TRAIL_MN:
        trailing_tables_block(a.qt, a.trail_k, nullptr, a.MN, nullptr, part64, part32);
        break;
    case ROLE_TRAIL_MX:
        trailing_tables_block(a.qt, a.trail_k, nullptr, nullptr, a.MX, part64, part32);
        break;
    }
}

// Leaf-count tables up to this size are staged in shared memory by the planner.
constexpr size_t PLAN_SMEM_MAX = 160 * 1024;

// The slice planner (Sec. 4, the role of Algorithm 4.1): S_req slices, or with
// auto_s as many as keep about min_leaves leaves per slice (at most S_req);
// writes the count and every slice's start (its first leaf, found by
// thread_unrank on the exact leaf counts W).  One thread per slice, grid-stride.
FS_D void plan_slices(const QueryConst& q, const Scratch& sc, const uint64_t* W, const int32_t* hs,
                      const Div32* dvh, uint64_t S_req, int auto_s, uint64_t min_leaves)
{
    const uint64_t L = total_leaves(q, W);
    uint64_t S = S_req;
    if (auto_s) {
        uint64_t want = (L + min_leaves - 1) / min_leaves;
        if (want < 1) want = 1;
        if (want < S) S = want;
    }
    // one division per block, shared
    __shared__ SliceSplit ssp;
    if (threadIdx.x == 0) {
        ssp = make_split(L, S, auto_s);
        if (blockIdx.x == 0) {
            sc.ctr[CTR_SEFF] = S;
            sc.ctr[CTR_L] = L;
            record_split(sc.ctr, ssp);
        }
    }
    __syncthreads();
    const SliceSplit split = ssp;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += nt) {
        int32_t* st = sc.starts + s * START_W;
        const uint64_t k0 = split.start(s);
        if (k0 >= L) {
            st[START_W - 1] = -1;
            continue;
        }
        int32_t pr;
        st[START_W - 1] = thread_unrank(q, hs, dvh, W, k0, pr,
                                        [&](int k, int32_t, int32_t a) { st[k] = a; });
    }
}

__global__ void __launch_bounds__(256) k_plan(const __grid_constant__ QueryConst q, Scratch sc,
                                              uint64_t S_req, int auto_s, uint64_t min_leaves)
{
    __shared__ int32_t hs[FS_MAX_D];
    __shared__ Div32 dvh[FS_MAX_D];
    if (threadIdx.x < FS_MAX_D) {
        hs[threadIdx.x] = q.h[threadIdx.x];
        dvh[threadIdx.x] = q.dv_h[threadIdx.x];
    }
    __syncthreads();
    plan_slices(q, sc, sc.W, hs, dvh, S_req, auto_s, min_leaves);
}

// The same with the leaf-count tables staged in shared memory (when they
// fit): one block per SM copies W once; its warps' probes then hit shared
// memory instead of L2.
__global__ void __launch_bounds__(1024) k_plan_smem(const __grid_constant__ QueryConst q, Scratch sc,
                                                    uint64_t S_req, int auto_s, uint64_t min_leaves)
{
    __shared__ int32_t hs[FS_MAX_D];
    __shared__ Div32 dvh[FS_MAX_D];
    extern __shared__ __align__(16) unsigned char dyn[];
    uint64_t* Ws = (uint64_t*)dyn;
    if (threadIdx.x < FS_MAX_D) {
        hs[threadIdx.x] = q.h[threadIdx.x];
        dvh[threadIdx.x] = q.dv_h[threadIdx.x];
    }
    if (blockIdx.x > 0) {  // a block with no slice (one per thread) skips the copy
        uint64_t S = S_req;
        if (auto_s) {
            const uint64_t want = (total_leaves(q, sc.W) + min_leaves - 1) / min_leaves;
            S = want < S ? (want < 1 ? 1 : want) : S;
        }
        if ((uint64_t)blockIdx.x * blockDim.x >= S) return;
    }
    const uint32_t words = (uint32_t)q.nw * (uint32_t)(q.n + 1);
    const ulonglong2* src = (const ulonglong2*)sc.W;  // 256-byte aligned section
    ulonglong2* dst = (ulonglong2*)Ws;
    // four independent 16-byte loads in flight per thread before their stores:
    // one block's copy is bound by the loads it keeps outstanding
    const uint32_t n2 = words / 2, bd = blockDim.x;
    for (uint32_t i = threadIdx.x; i < n2; i += 4 * bd) {
        ulonglong2 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (i + k * bd < n2) v[k] = src[i + k * bd];
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (i + k * bd < n2) dst[i + k * bd] = v[k];
    }
    if ((words & 1) && threadIdx.x == 0) Ws[words - 1] = sc.W[words - 1];
    __syncthreads();
    plan_slices(q, sc, Ws, hs, dvh, S_req, auto_s, min_leaves);
}

// off[s] = sum_{j < s} cnt[j] for s = 0..S (S = the planner's slice count),
// total -> ctr[CTR_TOTAL] and (optionally) *dev_count.  One block, tiles of
// 8 x blockDim slices: each thread loads 8 consecutive counts with four 16-byte
// vector loads (all of a tile's loads in flight at once), scans them in
// registers, and a warp-shuffle block scan of the thread totals places them.
__global__ void __launch_bounds__(1024) k_scan_slices(const uint64_t* cnt, uint64_t* off,
                                                      uint64_t* ctr, uint64_t* dev_count)
{
    __shared__ uint64_t wsum[32];
    const uint64_t S = ctr[CTR_SEFF];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nwarp = blockDim.x >> 5;
    const uint64_t tile = 8ull * blockDim.x;
    uint64_t carry = 0;
    for (uint64_t base = 0; base < S; base += tile) {
        const uint64_t i0 = base + 8ull * (uint64_t)tid;
        uint64_t v[8];
        if (i0 + 8 <= S) {
            const ulonglong2* p = (const ulonglong2*)(cnt + i0);  // 64-byte aligned
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const ulonglong2 x = p[k];
                v[2 * k] = x.x;
                v[2 * k + 1] = x.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = i0 + k < S ? cnt[i0 + k] : 0;
        }
        uint64_t sum = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) sum += v[k];
        uint64_t x = sum;  // inclusive scan of the thread totals within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint64_t y = lane < nwarp ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t t = __shfl_up_sync(FULL, y, o);
                if (lane >= o) y += t;
            }
            if (lane < nwarp) wsum[lane] = y;
        }
        __syncthreads();
        uint64_t run = carry + (w > 0 ? wsum[w - 1] : 0) + x - sum;
        if (i0 + 8 <= S) {
            uint64_t o[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                o[k] = run;
                run += v[k];
            }
            ulonglong2* q = (ulonglong2*)(off + i0);
#pragma unroll
            for (int k = 0; k < 4; k++) q[k] = make_ulonglong2(o[2 * k], o[2 * k + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++)
                if (i0 + k < S) {
                    off[i0 + k] = run;
                    run += v[k];
                }
        }
        carry += wsum[nwarp - 1];
        __syncthreads();  // wsum is rewritten by the next tile
    }
    if (tid == 0) {
        off[S] = carry;
        ctr[CTR_TOTAL] = carry;
        if (dev_count) *dev_count = carry;
    }
}

// hist[l] = sum_{j >= 0} D[l - j s] for l = 0..maxlen (s = |delta| for the
// strided difference array of the PAIR walk; s = 0 means D already is the
// histogram, as the PLAIN walk writes it).  In place on D, then copied to `hist` if given.
// Finishes the histogram (a strided prefix sum of the difference array when
// s > 0), copies it to the caller, and takes the count, the minimum and the
// maximum length from it into the call's counters.
__global__ void __launch_bounds__(1024) k_len_finalize(const __grid_constant__ QueryConst q,
                                                       uint64_t* D, uint64_t* hist, int s,
                                                       uint64_t* ctr)
{
    __shared__ uint64_t part[1024];
    __shared__ uint64_t wsum[32];
    __shared__ uint32_t wmin[32], wmax[32];
    const int len = q.maxlen + 1;
    if (s > 0) block_strided_prefix_sum(D, q.dv_in, D, len, s, part);
    uint64_t sum = 0;
    uint32_t mn = 0xffffffffu, mx = 0;
    for (int l = threadIdx.x; l < len; l += blockDim.x) {
        const uint64_t v = D[l];
        if (hist) hist[l] = v;
        if (v) {
            sum += v;
            mn = min(mn, (uint32_t)l);
            mx = max(mx, (uint32_t)l);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(FULL, sum, o);
        mn = min(mn, __shfl_xor_sync(FULL, mn, o));
        mx = max(mx, __shfl_xor_sync(FULL, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        wsum[w] = sum;
        wmin[w] = mn;
        wmax[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; k++) {
            sum += wsum[k];
            mn = min(mn, wmin[k]);
            mx = max(mx, wmax[k]);
        }
        ctr[CTR_COUNT] = sum;
        ctr[CTR_MINC] = sum ? 0xffffffffull - mn : 0ull;
        ctr[CTR_MAX] = sum ? mx : 0u;
    }
}

__global__ void k_copy_u64(const uint64_t* src, uint64_t* dst) { *dst = *src; }

// count, min and max of a length call from its counters to the caller's memory
__global__ void k_len_summary(const uint64_t* ctr, uint64_t* out)
{
    const uint64_t c = ctr[CTR_COUNT];
    out[0] = c;
    out[1] = c ? 0xffffffffull - ctr[CTR_MINC] : 0ull;
    out[2] = c ? ctr[CTR_MAX] : 0ull;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_precompute(const QueryConst& q, const Scratch& sc, cudaStream_t st,
                              const QueryConst* qt, int trail_k, uint64_t* T, int32_t* MN,
                              int32_t* MX)
{
    PrecompArgs a;
    memset(&a, 0, sizeof a);
    a.qw = q;
    if (qt) a.qt = *qt;
    a.W = sc.W;
    a.E = q.tab_e ? sc.E : nullptr;
    a.X0 = q.tab_xy ? sc.X0 : nullptr;
    a.YD = q.tab_xy ? sc.YD : nullptr;
    a.T = T;
    a.MN = MN;
    a.MX = MX;
    a.tmax = sc.ctr + CTR_TMAX;
    a.trail_k = trail_k;
    if (q.nw > 0) a.role[a.nroles++] = ROLE_WEIGHTS;
    if (q.tab_e || q.tab_xy) a.role[a.nroles++] = ROLE_PAIRTAB;
    if (qt && trail_k > 0) {
        a.role[a.nroles++] = ROLE_TRAIL;
        if (MN) a.role[a.nroles++] = ROLE_TRAIL_MN;
        if (MX) a.role[a.nroles++] = ROLE_TRAIL_MX;
    }
    if (a.nroles == 0) return cudaSuccess;
    k_precompute<<<a.nroles, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan_slices(const Scratch& sc, uint64_t* dev_count, cudaStream_t st)
{
    k_scan_slices<<<1, 1024, 0, st>>>(sc.slice_cnt, sc.slice_off, sc.ctr, dev_count);
    return cudaGetLastError();
}

cudaError_t launch_plan(const QueryConst& q, const Scratch& sc, uint64_t S_req, int auto_s,
                        uint64_t min_leaves, cudaStream_t st)
{
    const size_t wbytes = (size_t)q.nw * (size_t)(q.n + 1) * 8;
    if (wbytes > 0 && wbytes <= PLAN_SMEM_MAX && S_req >= 1024) {
        int sms = 0;
        cudaError_t e = sm_count_cached(&sms);
        if (e == cudaSuccess) e = smem_optin((const void*)k_plan_smem, (int)wbytes);
        if (e != cudaSuccess) return e;
        const uint64_t need = (S_req + 1023) / 1024;  // one slice per thread, one block per SM
        const unsigned blocks = (unsigned)(need < (uint64_t)sms ? need : (uint64_t)sms);
        k_plan_smem<<<blocks, 1024, wbytes, st>>>(q, sc, S_req, auto_s, min_leaves);
        return cudaGetLastError();
    }
    uint64_t blocks = (S_req + 255) / 256;  // one thread per slice
    if (blocks > 16384) blocks = 16384;
    if (blocks < 1) blocks = 1;
    k_plan<<<(unsigned)blocks, 256, 0, st>>>(q, sc, S_req, auto_s, min_leaves);
    return cudaGetLastError();
}

cudaError_t launch_len_finalize(const QueryConst& q, const Scratch& sc, uint64_t* hist, int s,
                                cudaStream_t st)
{
    k_len_finalize<<<1, 1024, 0, st>>>(q, sc.D, hist, s, sc.ctr);
    return cudaGetLastError();
}

cudaError_t launch_len_summary(const Scratch& sc, uint64_t* out, cudaStream_t st)
{
    k_len_summary<<<1, 1, 0, st>>>(sc.ctr, out);
    return cudaGetLastError();
}

cudaError_t launch_copy_u64(const uint64_t* src, uint64_t* dst, cudaStream_t st)
{
    k_copy_u64<<<1, 1, 0, st>>>(src, dst);
    return cudaGetLastError();
}

}  // namespace fsi
