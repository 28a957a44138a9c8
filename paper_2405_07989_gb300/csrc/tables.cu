// Per-query precompute and finalisation kernels.
//
//  k_pair_tables  the pair tables E / X0 / YD indexed by r mod lcm(A, B)
//                 (closed form of the congruence step, Sec. 3.2.4)
//  k_weights      the exact leaf counts W_k[p] that the slice planner unranks
//                 (balanced division of labour, Sec. 4.1 and Sec. 6.2)
//  k_plan         the slice planner: slice count and each slice's start state
//  k_scan_slices  exclusive scan of per-slice counts -> output offsets
//  k_len_finalize histogram from the strided difference array
#include "launch.h"
#include "walk.cuh"

namespace fsi {

// For w in [0, lcm): is w = x A + y B solvable with x, y >= 0 "within one
// period", and where the solutions of r = q lcm + w start (see pair_count).
__global__ void k_pair_tables(const __grid_constant__ QueryConst q, int8_t* E, int32_t* X0,
                              int32_t* YD)
{
    pair_tables_fill(q, E, X0, YD, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// W_k[p] = #{(a_k..a_{P-1}) >= 0 : sum_{i >= k} a_i h_i <= p} for k = 0..P-2,
// p = 0..n.  W_k = W_{k+1} / (1 - x^{h_k}) as series, i.e. a strided prefix
// sum; W_{P-1}[p] = floor(p / h_{P-1}) + 1 in closed form.  One block.
__global__ void __launch_bounds__(1024) k_weights(const __grid_constant__ QueryConst q,
                                                  uint64_t* W)
{
    __shared__ uint64_t part[1024];
    const int len = q.n + 1;
    for (int k = q.P - 2; k >= 0; k--) {
        const uint64_t* in = (k == q.P - 2) ? nullptr : W + (size_t)(k + 1) * len;
        block_strided_prefix_sum(in, q.dv_in, W + (size_t)k * len, len, q.h[k], part);
    }
}

// The slice planner (Sec. 4, the role of Algorithm 4.1): S_req slices, or with
// auto_s as many as keep about min_leaves leaves per slice (at most S_req);
// writes the count and every slice's start (its first leaf, found by
// warp_unrank on the exact leaf counts).  One warp per slice.
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
    const uint64_t L = total_leaves(q, sc.W);
    uint64_t S = S_req;
    if (auto_s) {
        uint64_t want = (L + min_leaves - 1) / min_leaves;
        if (want < 1) want = 1;
        if (want < S) S = want;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc.ctr[CTR_SEFF] = S;
        sc.ctr[CTR_L] = L;
    }
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const SliceSplit split(L, S);
    for (uint64_t s = gw; s < S; s += nw) {
        int32_t* st = sc.starts + s * START_W;
        const uint64_t k0 = split.start(s);
        if (k0 >= L) {
            if (lane == 0) st[START_W - 1] = -1;
            continue;
        }
        RunPrefix rp;
        const int32_t b = warp_unrank(q, hs, dvh, sc.W, k0, lane, rp);
        if (lane < q.P - 1) st[lane] = rp.a;
        if (lane == 0) st[START_W - 1] = b;
    }
}

// off[s] = sum_{j < s} cnt[j] for s = 0..S (S = the planner's slice count),
// total -> ctr[CTR_TOTAL] and (optionally) *dev_count.  One block; each thread
// sums a contiguous run of slices, then a block scan of the runs.
__global__ void __launch_bounds__(1024) k_scan_slices(const uint64_t* cnt, uint64_t* off,
                                                      uint64_t* ctr, uint64_t* dev_count)
{
    __shared__ uint64_t part[1024];
    const uint64_t S = ctr[CTR_SEFF];
    const int T = blockDim.x, tid = threadIdx.x;
    const uint64_t per = (S + T - 1) / T;
    const uint64_t b = (uint64_t)tid * per;
    const uint64_t e = b + per < S ? b + per : S;
    uint64_t s = 0;
#pragma unroll 8
    for (uint64_t i = b; i < e; i++) s += cnt[i];
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        uint64_t v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint64_t run = tid > 0 ? part[tid - 1] : 0;
    for (uint64_t i = b; i < e; i++) {
        off[i] = run;
        run += cnt[i];
    }
    if (tid == T - 1) {
        off[S] = part[T - 1];
        ctr[CTR_TOTAL] = part[T - 1];
        if (dev_count) *dev_count = part[T - 1];
    }
}

// hist[l] = sum_{j >= 0} D[l - j s] for l = 0..maxlen (s = |delta| for the
// strided difference array of the PAIR walk; s = 0 means D already is the
// histogram, as the PLAIN walk writes it).  In place on D, then copied to `hist` if given.
__global__ void __launch_bounds__(1024) k_len_finalize(const __grid_constant__ QueryConst q,
                                                       uint64_t* D, uint64_t* hist, int s)
{
    __shared__ uint64_t part[1024];
    const int len = q.maxlen + 1;
    if (s > 0) block_strided_prefix_sum(D, q.dv_in, D, len, s, part);
    if (hist)
        for (int l = threadIdx.x; l < len; l += blockDim.x) hist[l] = D[l];
}

__global__ void k_copy_u64(const uint64_t* src, uint64_t* dst) { *dst = *src; }

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
// length range.  One block.
__global__ void __launch_bounds__(1024) k_trailing_tables(const __grid_constant__ QueryConst q, int k,
                                                          uint64_t* T, int32_t* MN, int32_t* MX)
{
    __shared__ uint64_t part64[1024];
    __shared__ int32_t part32[1024];
    trailing_tables_block(q, k, T, MN, MX, part64, part32);
}

cudaError_t launch_trailing_tables(const QueryConst& q, int k, uint64_t* T, int32_t* MN, int32_t* MX,
                                   cudaStream_t st)
{
    k_trailing_tables<<<1, 1024, 0, st>>>(q, k, T, MN, MX);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_precompute(const QueryConst& q, const Scratch& sc, cudaStream_t st)
{
    if (q.tab_e || q.tab_xy) {
        int threads = 256;
        int blocks = (int)((q.lcm + threads - 1) / threads);
        if (blocks > 1024) blocks = 1024;
        k_pair_tables<<<blocks, threads, 0, st>>>(q, q.tab_e ? sc.E : nullptr,
                                                  q.tab_xy ? sc.X0 : nullptr,
                                                  q.tab_xy ? sc.YD : nullptr);
    }
    if (q.nw > 0) k_weights<<<1, 1024, 0, st>>>(q, sc.W);
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
    uint64_t blocks = (S_req + 7) / 8;  // one warp per slice
    if (blocks > 16384) blocks = 16384;
    if (blocks < 1) blocks = 1;
    k_plan<<<(unsigned)blocks, 256, 0, st>>>(q, sc, S_req, auto_s, min_leaves);
    return cudaGetLastError();
}

cudaError_t launch_len_finalize(const QueryConst& q, const Scratch& sc, uint64_t* hist, int s,
                                cudaStream_t st)
{
    k_len_finalize<<<1, 1024, 0, st>>>(q, sc.D, hist, s);
    return cudaGetLastError();
}

cudaError_t launch_copy_u64(const uint64_t* src, uint64_t* dst, cudaStream_t st)
{
    k_copy_u64<<<1, 1, 0, st>>>(src, dst);
    return cudaGetLastError();
}

}  // namespace fsi
