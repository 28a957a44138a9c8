// Enumerate write walk specialised for the common shapes: D = 3..8 levels,
// the pair resolved through its tables, and the caller's column order equal to
// the walk order or its reverse (generators given in descending or ascending
// order).  A row's values are assembled in registers in caller order and
// stored with fixed offsets (8-byte stores where the row is aligned).  Each
// lane writes the rows of its own leaf, at the position the warp's scan of
// row counts gives it: no row-to-leaf search and no shuffles per row (the
// lanes of a chunk differ in row count by a few rows, so the divergent loop
// stays short).  64 registers, four 256-thread blocks per SM.
// Same results, layout and staging as the generic walk in enum.cu.
#include "enum_common.cuh"
#include "launch.h"

namespace fsi {

// A chunk whose leaves all have at most this many rows is written one lane per
// leaf; otherwise leaf by leaf with all lanes.
constexpr uint32_t LEAF_ROWS_MAX = 64;

// PERM 1: caller column of level k is D-1-k; PERM 2: it is k.
template <typename ELEM, int D, int PERM>
struct EnumFix {
    static constexpr int NP = D - 3;  // run-prefix levels
    Stager<ELEM> sg;
    const int32_t* X0;
    const int32_t* YD;
    const uint64_t* slice_off;
    const uint64_t* blk;
    uint64_t* ctr;
    int32_t pre[NP > 0 ? NP : 1];
    int32_t a2base, lpbase;  // level P-2 and prefix sum of the sibling group's first run

    static constexpr bool SKIP = true;
    static constexpr bool ANY_ORDER = false;
    FS_D void fault() { flag_fault(ctr); }
    FS_D void group_begin(const QueryConst&, const RunPrefix& rp, int, int32_t ac, int32_t lpc)
    {
#pragma unroll
        for (int k = 0; k < NP - 1; k++) pre[k] = __shfl_sync(FULL, rp.a, k);
        a2base = ac;
        lpbase = lpc;
    }
    // level P-2 of this lane's leaf
    FS_D int32_t level2(int32_t lp) const
    {
        if constexpr (NP == 0) return 0;
        else return a2base + (lp - lpbase);
    }
    FS_D void slice_begin(const QueryConst&, uint64_t s)
    {
        sg.begin(slice_off[s] + (blk ? blk[s / SLICE_GROUP] : 0ull));
    }
    FS_D void slice_end(const QueryConst&, uint64_t) { sg.flush(); }

    FS_D void put_row(ELEM* row, int32_t a2, int32_t a, int32_t x, int32_t y) const
    {
        int32_t lev[D];
#pragma unroll
        for (int k = 0; k < NP; k++) lev[k] = k == NP - 1 ? a2 : pre[k];
        lev[NP] = a;
        lev[NP + 1] = x;
        lev[NP + 2] = y;
        int32_t val[D];
#pragma unroll
        for (int c = 0; c < D; c++) val[c] = lev[PERM == 1 ? D - 1 - c : c];
        if constexpr (D % 2 == 0 && sizeof(ELEM) == 4) {
#pragma unroll
            for (int m = 0; m < D / 2; m++)
                *reinterpret_cast<int2*>(row + 2 * m) = make_int2(val[2 * m], val[2 * m + 1]);
        } else if constexpr (D % 2 == 0 && sizeof(ELEM) == 2) {
#pragma unroll
            for (int m = 0; m < D / 2; m++)
                *reinterpret_cast<uint32_t*>(row + 2 * m) =
                    (uint32_t)(uint16_t)val[2 * m] | ((uint32_t)(uint16_t)val[2 * m + 1] << 16);
        } else {
#pragma unroll
            for (int c = 0; c < D; c++) row[c] = (ELEM)val[c];
        }
    }

    // The rows of the leaf in lane `src`, all lanes together: for chunks with a
    // leaf of more than LEAF_ROWS_MAX rows, where one lane per leaf would idle
    // the others.
    FS_D void emit_one(const QueryConst& q, int lane, uint32_t cs, int32_t xs, int32_t ys,
                       int32_t as, int32_t a2s)
    {
        for (uint32_t t0 = 0; t0 < cs;) {
            uint32_t room = sg.template room<D>();
            if (room == 0) {
                sg.flush();
                room = sg.template room<D>();
            }
            const uint32_t npc = min(room, cs - t0);
            ELEM* sb = sg.cursor();
            for (uint32_t j = 0; j < npc; j += 32) {
                const uint32_t k = j + lane;
                if (k < npc) {
                    const int32_t t = (int32_t)(t0 + k);
                    put_row(sb + k * D, a2s, as, xs + t * q.v, ys - t * q.u);
                }
            }
            sg.nst += (int32_t)npc;
            t0 += npc;
        }
    }

    FS_D bool chunk(const QueryConst& q, int lane, bool valid, int32_t r, int32_t a, int32_t lp)
    {
        const int32_t a2 = level2(lp);
        int32_t x0 = 0, y0 = 0;
        uint32_t c = 0;
        if (valid) c = pair_xy<true>(q, X0, YD, r, x0, y0);
        if (__any_sync(FULL, c > (uint32_t)LEAF_ROWS_MAX)) {
            for (int src = 0; src < 32; src++) {
                const uint32_t cs = __shfl_sync(FULL, c, src);
                const int32_t xs = __shfl_sync(FULL, x0, src);
                const int32_t ys = __shfl_sync(FULL, y0, src);
                const int32_t as = __shfl_sync(FULL, a, src);
                const int32_t a2s = __shfl_sync(FULL, a2, src);
                if (cs) emit_one(q, lane, cs, xs, ys, as, a2s);
            }
            return false;
        }
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t T = __shfl_sync(FULL, incl, 31);
        const uint32_t excl = incl - c;
        // the rows fill the staging buffer to its end before it is flushed
        for (uint32_t ps = 0; ps < T;) {
            uint32_t room = sg.template room<D>();
            if (room == 0) {
                sg.flush();
                room = sg.template room<D>();
            }
            const uint32_t npc = min(room, T - ps);
            ELEM* sb = sg.cursor();
            // this lane's rows of [ps, ps + npc): t = i - excl of its leaf
            const uint32_t lo = max(excl, ps), hi = min(incl, ps + npc);
            int32_t t = (int32_t)(lo - excl);
            for (uint32_t i = lo; i < hi; i++, t++)
                put_row(sb + (i - ps) * D, a2, a, x0 + t * q.v, y0 - t * q.u);
            sg.nst += (int32_t)npc;
            ps += npc;
        }
        return false;
    }
};

template <typename ELEM, int D, int PERM>
__global__ void __launch_bounds__(256, 4) k_pair_enum_fix(const __grid_constant__ QueryConst q,
                                                          Scratch sc, int queue, ELEM* out,
                                                          uint64_t cap_rows)
{
    __shared__ SmemQ sq;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq, sc.ctr);
    int32_t* X0 = (int32_t*)dyn;
    int32_t* YD = X0 + q.lcm;
    for (uint32_t i = threadIdx.x; i < q.lcm; i += blockDim.x) {
        X0[i] = sc.X0[i];
        YD[i] = sc.YD[i];
    }
    const size_t tab = ((size_t)q.lcm * 8 + 15) & ~(size_t)15;
    unsigned char* wp = dyn + tab + (size_t)(threadIdx.x >> 5) * ENUM_WARP_BYTES;
    __syncthreads();
    using C = EnumFix<ELEM, D, PERM>;
    C cons;
    cons.sg.out = out;
    cons.sg.cap_elems = cap_rows * (uint64_t)D;
    cons.sg.lo_elems = sc.row_lo * (uint64_t)D;
    cons.sg.wbase = wp;
    cons.sg.d = D;
    cons.sg.begin(0);
    cons.X0 = X0;
    cons.YD = YD;
    cons.slice_off = sc.slice_off;
    cons.blk = sc.blk;
    cons.ctr = sc.ctr;
#pragma unroll
    for (int k = 0; k < C::NP; k++) cons.pre[k] = 0;
    cons.a2base = 0;
    cons.lpbase = 0;
    run_queue(q, sq, sc, queue, cons);
    cons.sg.finish();
}

template <typename ELEM, int PERM>
static void* pick_d(int D)
{
    switch (D) {
    case 3: return (void*)k_pair_enum_fix<ELEM, 3, PERM>;
    case 4: return (void*)k_pair_enum_fix<ELEM, 4, PERM>;
    case 5: return (void*)k_pair_enum_fix<ELEM, 5, PERM>;
    case 6: return (void*)k_pair_enum_fix<ELEM, 6, PERM>;
    case 7: return (void*)k_pair_enum_fix<ELEM, 7, PERM>;
    case 8: return (void*)k_pair_enum_fix<ELEM, 8, PERM>;
    }
    return nullptr;
}

void* pair_enum_fixed_kernel(const QueryConst& q, int elem_bytes)
{
    if (!q.tab_xy || q.d != q.D || q.D > 8) return nullptr;
    bool rev = true, ident = true;
    for (int k = 0; k < q.D; k++) {
        rev = rev && q.col[k] == q.D - 1 - k;
        ident = ident && q.col[k] == k;
    }
    if (!rev && !ident) return nullptr;
    if (elem_bytes == 2) return rev ? pick_d<int16_t, 1>(q.D) : pick_d<int16_t, 2>(q.D);
    return rev ? pick_d<int32_t, 1>(q.D) : pick_d<int32_t, 2>(q.D);
}

}  // namespace fsi
