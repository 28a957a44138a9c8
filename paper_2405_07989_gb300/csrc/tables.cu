// Per-query precompute and finalisation kernels.
//
//  k_pair_tables  the pair tables E / X0 / YD indexed by r mod lcm(A, B)
//                 (closed form of the congruence step, Sec. 3.2.4)
//  k_weights      the exact leaf counts W_k[p] that the slice planner unranks
//                 (balanced division of labour, Sec. 4.1 and Sec. 6.2)
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
    const uint32_t lcm = q.lcm;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < lcm;
         w += gridDim.x * blockDim.x) {
        int8_t e = -1;
        int32_t x0 = -1, yd = 0;
        if (w % (uint32_t)q.G == 0) {
            uint64_t wg = w / (uint32_t)q.G;
            uint64_t x = ((wg % (uint64_t)q.v) * (uint64_t)q.inv) % (uint64_t)q.v;
            int64_t rest = (int64_t)w - (int64_t)x * q.A;  // divisible by B
            x0 = (int32_t)x;
            yd = (int32_t)(rest / q.B);
            e = rest >= 0 ? 1 : 0;
        }
        if (E) E[w] = e;
        if (X0) X0[w] = x0;
        if (YD) YD[w] = yd;
    }
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

// off[s] = sum_{j < s} cnt[j] for s = 0..S, total -> ctr[CTR_TOTAL] and
// (optionally) *dev_count.  One block.
__global__ void __launch_bounds__(1024) k_scan_slices(const uint64_t* cnt, uint64_t* off,
                                                      uint64_t S, uint64_t* ctr,
                                                      uint64_t* dev_count)
{
    __shared__ uint64_t part[1024];
    const int T = blockDim.x, tid = threadIdx.x;
    const uint64_t per = (S + T - 1) / T;
    const uint64_t b = (uint64_t)tid * per;
    const uint64_t e = b + per < S ? b + per : S;
    uint64_t s = 0;
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

cudaError_t launch_scan_slices(const Scratch& sc, uint64_t S, uint64_t* dev_count, cudaStream_t st)
{
    k_scan_slices<<<1, 1024, 0, st>>>(sc.slice_cnt, sc.slice_off, S, sc.ctr, dev_count);
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
