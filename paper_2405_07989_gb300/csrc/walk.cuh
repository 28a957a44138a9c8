// Device-side building blocks of the bounded lexicographic walk.
//
// The lex order on the leaves (prefixes (a_0..a_{P-1}) with phi <= n, walk
// order, a_0 most significant) is cut into S slices of consecutive leaf ranks
// (Sec. 4: a bound splits the lex-ordered output between workers; here the
// bounds are clean prefixes (leaf, 0, 0), so each worker's stream starts at a
// state that satisfies the hypothesis of Thm 3.2, cf. Remark 4.2).  A warp
// takes one slice at a time, finds the slice's first leaf from the exact leaf
// counts W (the planner), and then walks the slice's leaves in lex order, 32
// leaves per step: lane l takes the l-th next leaf.
#pragma once

#include <cuda_runtime.h>

#include "fs_internal.h"

namespace fsi {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Slices: slice s holds the leaf ranks [floor(s L / S), floor((s+1) L / S)).
// Written as s*Q + floor(s*R / S) with L = Q*S + R, exact for S < 2^32.
// ---------------------------------------------------------------------------
FS_HD uint64_t slice_start(uint64_t s, uint64_t L, uint64_t S)
{
    uint64_t Q = L / S, R = L % S;
    return s * Q + (s * R) / S;
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

FS_D void block_strided_prefix_sum(const uint64_t* in, const Div32& dv_in, uint64_t* out, int len,
                                   int s, uint64_t* part)
{
    const int T = blockDim.x, tid = threadIdx.x;
    if (len <= 0) return;
    if (s >= T || s >= len) {
        // many short chains: one thread per chain
        int nch = s < len ? s : len;
        for (int rho = tid; rho < nch; rho += T) {
            uint64_t sum = 0;
            for (int p = rho; p < len; p += s) {
                sum += sps_in(in, p, dv_in);
                out[p] = sum;
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
    int t0 = g * seg, t1 = t0 + seg;
    uint64_t sum = 0;
    if (act) {
        for (int t = t0; t < t1; t++) {
            long long p = rho + (long long)t * s;
            if (p >= len) break;
            sum += sps_in(in, (int)p, dv_in);
        }
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
    if (act) {
        for (int t = t0; t < t1; t++) {
            long long p = rho + (long long)t * s;
            if (p >= len) break;
            run += sps_in(in, (int)p, dv_in);
            out[p] = run;
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
// The slice walk.  Cons must provide
//   void run_loaded(const QueryConst&, int slot, const RunPrefix&, int lane)
//       -- a run's prefix was loaded into slot 0/1 (warp-uniform call);
//   bool chunk(const QueryConst&, int lane, bool valid, int32_t r, int32_t a,
//              int32_t lp, int slot)
//       -- one leaf per lane: residual r left for the pair, a = a_{P-1},
//          lp = length of the run prefix, slot of its run; returns true to
//          stop the walk (warp-uniform).
// Returns true if the consumer stopped the walk.
// ---------------------------------------------------------------------------
template <class Cons>
FS_D bool walk_slice(const QueryConst& q, const int32_t* hs, const Div32* dvh, const uint64_t* W,
                     uint64_t rank0, uint64_t nleaves, int lane, int32_t hk, Cons& cons)
{
    RunPrefix rp;
    int32_t b = warp_unrank(q, hs, dvh, W, rank0, lane, rp);
    const int np = q.P - 1;
    const int32_t hin = hs[q.P - 1];
    int32_t Rc = np > 0 ? __shfl_sync(FULL, rp.r, np - 1) : q.n;
    int32_t lpc = np > 0 ? __shfl_sync(FULL, rp.l, np - 1) : 0;
    int32_t lenc = (int32_t)div32((uint32_t)Rc, q.dv_in) + 1;
    int cs = 0;
    cons.run_loaded(q, 0, rp, lane);
    int32_t Rn = -1, lpn = 0, lenn = 0;
    if (warp_next_run(q, lane, hk, rp)) {
        Rn = __shfl_sync(FULL, rp.r, np - 1);
        lpn = __shfl_sync(FULL, rp.l, np - 1);
        lenn = (int32_t)div32((uint32_t)Rn, q.dv_in) + 1;
        cons.run_loaded(q, 1, rp, lane);
    }
    uint64_t rem = nleaves;
    for (;;) {
        // fast path: whole chunks inside the current run
        {
            int32_t k = lenc - b;
            uint64_t nfull = (uint64_t)(k >> 5);
            if (rem >> 5 < nfull) nfull = rem >> 5;
            if (nfull > 0) {
                int32_t a = b + lane;
                int32_t r = Rc - a * hin;
                const int32_t step = 32 * hin;
                for (uint64_t i = 0; i < nfull; i++) {
                    if (cons.chunk(q, lane, true, r, a, lpc, cs)) return true;
                    r -= step;
                    a += 32;
                }
                b += (int32_t)(nfull << 5);
                rem -= nfull << 5;
                if (rem == 0) return false;
            }
        }
        // general chunk: may span the end of the current run and the next run
        const int32_t k = lenc - b;  // >= 1 leaves left in the current run
        const bool inc = lane < k;
        int32_t a, r;
        if (inc) {
            a = b + lane;
            r = Rc - a * hin;
        } else {
            a = lane - k;
            r = (a < lenn) ? Rn - a * hin : -1;
        }
        int32_t avail = k >= 32 ? 32 : min(32, k + min(lenn, 32));
        int32_t nproc = (rem < (uint64_t)avail) ? (int32_t)rem : avail;
        if (nproc <= 0) {
            // the slice claims leaves past the last one: only a planner fault
            // can cause this; flag it and end the walk rather than spin
            cons.fault();
            return false;
        }
        const bool valid = lane < nproc;
        if (cons.chunk(q, lane, valid, r, a, inc ? lpc : lpn, inc ? cs : (cs ^ 1))) return true;
        rem -= (uint64_t)nproc;
        if (rem == 0) return false;
        if (nproc < k) {
            b += nproc;
            continue;
        }
        // the current run is finished: the next run becomes current
        const int32_t used = nproc - k;
        Rc = Rn;
        lpc = lpn;
        lenc = lenn;
        cs ^= 1;
        b = used;
        Rn = -1;
        lenn = 0;
        if (warp_next_run(q, lane, hk, rp)) {
            Rn = __shfl_sync(FULL, rp.r, np - 1);
            lpn = __shfl_sync(FULL, rp.l, np - 1);
            lenn = (int32_t)div32((uint32_t)Rn, q.dv_in) + 1;
            cons.run_loaded(q, cs ^ 1, rp, lane);
        }
        if (b == lenc) {
            // that run was consumed entirely by this chunk
            Rc = Rn;
            lpc = lpn;
            lenc = lenn;
            cs ^= 1;
            b = 0;
            Rn = -1;
            lenn = 0;
            if (warp_next_run(q, lane, hk, rp)) {
                Rn = __shfl_sync(FULL, rp.r, np - 1);
                lpn = __shfl_sync(FULL, rp.l, np - 1);
                lenn = (int32_t)div32((uint32_t)Rn, q.dv_in) + 1;
                cons.run_loaded(q, cs ^ 1, rp, lane);
            }
        }
    }
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
template <bool TAB>
FS_D uint32_t pair_count(const QueryConst& q, const int8_t* E, int32_t r)
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
        uint32_t x0 = (uint32_t)(((uint64_t)t * (uint32_t)q.inv) % (uint32_t)q.v);
        uint32_t xmax = div32((uint32_t)r, q.dv_A);
        return xmax >= x0 ? div32(xmax - x0, q.dv_v) + 1u : 0u;
    }
}

template <bool TAB>
FS_D uint32_t pair_xy(const QueryConst& q, const int32_t* X0, const int32_t* YD, int32_t r,
                      int32_t& x0, int32_t& y0)
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
        uint32_t xx = (uint32_t)(((uint64_t)t * (uint32_t)q.inv) % (uint32_t)q.v);
        uint32_t xmax = div32((uint32_t)r, q.dv_A);
        if (xmax < xx) return 0u;
        x0 = (int32_t)xx;
        y0 = (int32_t)div32((uint32_t)(r - (int32_t)xx * q.A), q.dv_B);
        return div32(xmax - xx, q.dv_v) + 1u;
    }
}

// warp sums
FS_D uint64_t warp_sum_u64(uint64_t v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

}  // namespace fsi
