// Internal definitions shared by the CUDA translation units of the library.
//
// Walk layout.  The walk uses D = max(d, 3) "levels".  Levels 0..P-1 (P = D-2)
// are the prefix levels: a prefix (a_0..a_{P-1}) with phi <= n is a LEAF.  Levels
// P and P+1 hold the pair (A, B) that the PAIR method resolves in closed form.
// Level P-1 is the innermost prefix level; the prefixes of levels 0..P-2 are
// RUNS (a run is the sequence of leaves a_{P-1} = 0, 1, ... under one run
// prefix).  For d < 3, virtual levels with generator n+1 (so their coordinate is
// always 0) pad the walk to 3 levels; they have no output column.
#pragma once

#include <stdint.h>

#include "../../include/fs.h"

#if defined(__CUDACC__)
#define FS_HD __host__ __device__ __forceinline__
#define FS_D __device__ __forceinline__
#else
#define FS_HD inline
#define FS_D inline
#endif

namespace fsi {

// ---------------------------------------------------------------------------
// Division by an invariant divisor.
//
// Granlund & Montgomery, "Division by invariant integers using multiplication"
// (PLDI 1994), Thm 4.2: if 2^(N+l) <= m*dv <= 2^(N+l) + 2^l then
// floor(x/dv) = floor(m*x / 2^(N+l)) for all 0 <= x < 2^N.  With N = 31,
// l = ceil(log2 dv) and m = ceil(2^(31+l) / dv) both inequalities hold and
// m < 2^32.  Since x < 2^31, floor(m x / 2^(31+l)) = floor(m (2x) / 2^(32+l))
// = (high word of m * 2x) >> l: a multiply-high and a 32-bit shift.
// ---------------------------------------------------------------------------
struct Div32 {
    uint32_t m;
    uint32_t l;   // ceil(log2 dv)
    uint32_t dv;
};

inline Div32 make_div32(uint32_t dv)
{
    uint32_t l = 0;
    while (l < 32 && ((uint64_t)1 << l) < dv) l++;
    Div32 r;
    r.l = l;
    r.m = (uint32_t)((((uint64_t)1 << (31 + l)) + dv - 1) / dv);
    r.dv = dv;
    return r;
}

FS_HD uint32_t div32(uint32_t x, const Div32& q)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(x + x, q.m) >> q.l;
#else
    return (uint32_t)(((uint64_t)(x + x) * q.m) >> 32) >> q.l;
#endif
}

// ---------------------------------------------------------------------------
// Per-query constants, computed on the host from (n, g) and passed to every
// kernel by value.  Tables that depend on n (leaf weights) or on lcm(A, B)
// (pair tables) are built on the device from these constants.
// ---------------------------------------------------------------------------
enum { TABLE_E_MAX = 16384, TABLE_XY_MAX = 4096 };
// "no solution" bound of the trailing-three length tables
enum { TRIPLE_NONE = 1 << 30 };

struct QueryConst {
    int32_t n;            // the element
    int32_t d;            // caller's dimension
    int32_t D;            // walk levels, max(d, 3)
    int32_t P;            // prefix levels, D - 2 (>= 1)
    int32_t h[FS_MAX_D];  // generator of each walk level
    int32_t col[FS_MAX_D];// caller column of each walk level, -1 for a virtual level
    // the pair: A = h[P], B = h[P+1]
    int32_t A, B;
    int32_t G;            // gcd(A, B)
    int32_t u, v;         // A / G, B / G
    int32_t inv;          // u^-1 mod v (0 if v == 1)
    int32_t delta;        // v - u: change of a_P + a_{P+1} per step t of the pair
    uint32_t lcm;         // lcm(A, B) when a table path is possible, else 0
    int32_t tab_e;        // 1: the count table E[lcm] is used
    int32_t tab_xy;       // 1: the tables X0[lcm], YD[lcm] are used
    Div32 dv_lcm, dv_in, dv_A, dv_B, dv_G, dv_v;
    Div32 dv_h[FS_MAX_D]; // per level, for the PLAIN method's decrementAndSolve
    int32_t maxlen;       // floor(n / min real g): the largest possible length
    int32_t dbins;        // histogram difference-array size: maxlen + |delta| + 1
    int32_t nw;           // number of leaf-weight tables: P - 1
    // Common-divisor skipping (the congruence of Sec. 3.2.4 over the generators
    // after the walk's innermost level): a leaf's residual R - a h_in must be a
    // multiple of Gt, the gcd of those generators, for any completion to
    // exist.  That holds iff sk_g = gcd(h_in, Gt) divides R and
    // a = (R / sk_g) sk_inv (mod sk_m), sk_m = Gt / sk_g, sk_inv =
    // (h_in / sk_g)^-1 mod sk_m; the walk visits only that class.  Index 0 is
    // the walk's own query, 1 and 2 the trailing-three / trailing-four walks
    // (reduce_to_trailing moves them to 0).  sk_g = sk_m = 1: nothing skipped.
    int32_t sk_g[3], sk_m[3], sk_inv[3];
    Div32 dv_skg[3], dv_skm[3];
    int32_t walk;         // fs_walk: how the order-free walks take a sibling group
    // The pair count of one lane over one sibling group fits 32 bits: a lane
    // takes at most 32 (n / h_in + 1) leaves of a group and each has at most
    // n / lcm + 1 completions (PAIR count walk; set by build_query).
    int32_t acc32;
    // floor(x / lcm) = umulhi(x, lcm_m1) for every residual x <= n when fdiv:
    // with lcm_m1 = ceil(2^32 / lcm) = (2^32 + e) / lcm, 0 <= e < lcm, the
    // product x lcm_m1 / 2^32 exceeds x / lcm by x e / (lcm 2^32) < 1 / lcm
    // while n lcm < 2^32, too little to reach the next integer (set by
    // build_query for lcm >= 2).
    uint32_t lcm_m1;
    int32_t fdiv;
};

// ---------------------------------------------------------------------------
// Device scratch layout of one call (byte offsets into the scratch arena).
// ---------------------------------------------------------------------------
// Slices counted per block when enumerate's first walk goes run by run (the
// groups of Scratch::blk).
constexpr int SLICE_GROUP = 32;

enum Ctr {
    CTR_QUEUE = 0,    // slice queue head (first walk)
    CTR_QUEUE2 = 1,   // slice queue head (second walk)
    CTR_COUNT = 2,    // total count
    CTR_FOUND = 3,    // predicate found flag
    CTR_MINC = 4,     // UINT32_MAX - min length (atomicMax)
    CTR_MAX = 5,      // max length (atomicMax)
    CTR_ERR = 6,      // error flags
    CTR_TOTAL = 7,    // enumerate: total rows (from the scan)
    CTR_SEFF = 8,     // number of slices the planner chose
    CTR_L = 9,        // number of leaves
    CTR_DONE = 10,    // blocks of a count walk that have added their part
    CTR_SQ = 11,      // leaves per head slice (planner; SliceSplit::Q)
    CTR_SR = 12,      // head slices with one leaf more (SliceSplit::R)
    CTR_TMAX = 13,    // largest entry of the trailing count table (precompute)
    CTR_SH = 14,      // head slices (SliceSplit::Sh)
    CTR_LH = 15,      // leaves of the head slices (SliceSplit::Lh)
    CTR_TQ = 16,      // leaves per tail slice (SliceSplit::Qt)
    CTR_TR = 17,      // tail slices with one leaf more (SliceSplit::Rt)
    CTR_N = 24
};

struct Scratch {
    uint64_t* ctr;        // CTR_N counters
    uint64_t* W;          // nw * (n + 1) leaf weights
    int8_t* E;            // lcm
    int32_t* X0;          // lcm
    int32_t* YD;          // lcm
    uint64_t* slice_cnt;  // S
    uint64_t* slice_off;  // S + 1 row offsets; with blk: offsets within a group of 32 slices
    uint64_t* blk;        // NULL, or the row offset of each group of SLICE_GROUP
                          // slices: slice s starts at row blk[s / SLICE_GROUP] + slice_off[s]
    uint64_t* D;          // dbins (global difference array)
    int32_t* starts;      // S * FS_MAX_D slice start states (planner output)
    // the window a walk covers: slices [s_lo, min(S, s_hi)); an enumerate
    // writes global row g to row g - row_lo of its buffer (rows outside
    // [row_lo, row_lo + cap) are dropped)
    uint64_t s_lo, s_hi, row_lo;
};

// ---------------------------------------------------------------------------
// Batched queries (batch.cu)
// ---------------------------------------------------------------------------
struct BatchQ {
    QueryConst q;
    uint64_t off_W, off_E, off_X0, off_YD;  // byte offsets of its tables in the arena
    uint64_t off_T3, off_MN3, off_MX3;      // trailing-k tables (trail = k)
    uint64_t L;      // leaves of the walk (device)
    uint64_t S;      // slices (device)
    uint64_t item0;  // first work item (device)
    int32_t valid;   // 0: invalid query, skipped
    int32_t trail;   // k = 3 or 4: walk the first d-k levels, the last k from tables; 0: pair
};

struct BatchRes {
    unsigned long long count;
    unsigned long long minc;  // UINT32_MAX - min length (atomicMax)
    unsigned long long max;
};

enum BatchCtr { BCTR_QUEUE = 0, BCTR_ITEMS = 1, BCTR_ERR = 2, BCTR_N = 8 };

struct BatchDev {
    BatchQ* qs;
    int nq;
    int mode;               // 0: count; 1: count + min / max length
    unsigned char* arena;   // per-query tables
    int32_t* starts;        // items_cap * START_W (slice, query, start state)
    uint64_t items_cap;
    uint64_t items_target;
    uint64_t min_leaves;
    uint64_t* ctr;          // BCTR_N counters
    BatchRes* res;          // nq results
};

// Predicate constants for the ANY consumer.
struct PredConst {
    int64_t w[FS_MAX_D];  // weight of each walk level (0 for virtual levels)
    int64_t c;
    int32_t op;
    int32_t modulus;      // 0: comparison; else congruence
    // pair: value changes by dw per step t of the pair
    int64_t dw;
    // congruence data: g = gcd(dw mod M, M), Mq = M / g, invq = (dw/g)^-1 mod Mq
    int64_t gM, Mq, invq;
};

}  // namespace fsi
