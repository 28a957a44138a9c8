// Enumerate (the save consumer of Sec. 2), second walk of fs_enumerate.
//
// The first walk counted every slice; a scan turned the counts into row
// offsets, so each slice writes its rows into its own contiguous range
// [off_s, off_s + count_s) of the caller's buffer, in lex order.  Per chunk of
// 32 leaves: a warp scan of the per-leaf row counts, a row -> leaf map in
// shared memory, then one row per lane written into a shared-memory staging
// buffer.  Full staging buffers are drained to global memory by the bulk-copy
// engine (cp.async.bulk, 16-byte aligned body), the unaligned head and tail by
// plain stores; the warp waits for its copy to have read the buffer before
// refilling it (other warps run meanwhile).
#include "enum_common.cuh"
#include "launch.h"

namespace fsi {

// Generic write walk: any column order, any number of levels (MAXL = 4, 8:
// run prefixes and columns in registers; MAXL = 16: in shared memory), table
// or division path.  Row -> leaf through a map in shared memory.
template <bool TAB, typename ELEM, int MAXL>
struct EnumCons {
    static constexpr bool REGS = MAXL <= 8;
    static constexpr int NR = REGS ? MAXL - 3 : 1;  // run-prefix levels held in registers

    Stager<ELEM> sg;
    const int32_t* X0;
    const int32_t* YD;
    const uint64_t* slice_off;
    const uint64_t* blk;
    uint8_t* map;          // row -> lane of its leaf, ENUM_MAPCAP entries
    int32_t* tmpl;         // MAXL = 16: the current run's prefix by level
    const int32_t* scol;   // MAXL = 16: column of each level
    uint64_t* ctr;
    int32_t piece, np;
    int32_t cin, cA, cB;   // columns of level P-1 and of the pair (-1: virtual)
    int32_t col[NR];
    int32_t pre[NR];
    int32_t a2base, lpbase;  // level P-2 and prefix sum of the sibling group's first run

    static constexpr bool SKIP = true;
    static constexpr bool ANY_ORDER = false;
    FS_D void fault() { flag_fault(ctr); }

    // the levels above P-2 are the group's; level P-2 differs by lane (a2)
    FS_D void group_begin(const QueryConst&, const RunPrefix& rp, int lane, int32_t ac, int32_t lpc)
    {
        if constexpr (REGS) {
#pragma unroll
            for (int k = 0; k < NR; k++) {
                const int32_t v = __shfl_sync(FULL, rp.a, k);
                if (k < np - 1) pre[k] = v;
            }
        } else {
            __syncwarp();  // earlier rows have read the previous group's prefix
            if (lane < np - 1) tmpl[lane] = rp.a;
            __syncwarp();
        }
        a2base = ac;
        lpbase = lpc;
    }

    FS_D void slice_begin(const QueryConst&, uint64_t s)
    {
        sg.begin(slice_off[s] + (blk ? blk[s / SLICE_GROUP] : 0ull));
    }
    FS_D void slice_end(const QueryConst&, uint64_t) { sg.flush(); }

    // Rows [excl, incl) of this chunk belong to this lane's leaf; T rows in all.
    FS_D void emit(const QueryConst& q, int lane, uint32_t T, uint32_t excl, uint32_t incl,
                   int32_t x0, int32_t y0, int32_t a, int32_t a2)
    {
        const int d = sg.d;
        for (uint32_t ps = 0; ps < T; ps += (uint32_t)piece) {
            const uint32_t npc = min((uint32_t)piece, T - ps);
            if (!sg.fits((int)npc)) sg.flush();
            const uint32_t lo = max(excl, ps), hi = min(incl, ps + npc);
            for (uint32_t i = lo; i < hi; i++) map[i - ps] = (uint8_t)lane;
            __syncwarp();
            ELEM* sb = sg.cursor();
            for (uint32_t j = 0; j < npc; j += 32) {
                const uint32_t i = j + lane;
                const bool ok = i < npc;
                const int src = ok ? map[i] : 0;
                const uint32_t es = __shfl_sync(FULL, excl, src);
                const int32_t xs = __shfl_sync(FULL, x0, src);
                const int32_t ys = __shfl_sync(FULL, y0, src);
                const int32_t as = __shfl_sync(FULL, a, src);
                const int32_t a2s = __shfl_sync(FULL, a2, src);
                if (ok) {
                    const int32_t t = (int32_t)(ps + i - es);
                    ELEM* row = sb + i * d;
                    if constexpr (REGS) {
#pragma unroll
                        for (int k = 0; k < NR; k++)
                            if (k < np && col[k] >= 0) row[col[k]] = (ELEM)(k == np - 1 ? a2s : pre[k]);
                    } else {
                        for (int k = 0; k < np; k++) {
                            const int c = scol[k];
                            if (c >= 0) row[c] = (ELEM)(k == np - 1 ? a2s : tmpl[k]);
                        }
                    }
                    if (cin >= 0) row[cin] = (ELEM)as;
                    if (cA >= 0) row[cA] = (ELEM)(xs + t * q.v);
                    if (cB >= 0) row[cB] = (ELEM)(ys - t * q.u);
                }
            }
            sg.nst += (int32_t)npc;
            __syncwarp();
        }
    }

    FS_D bool chunk(const QueryConst& q, int lane, bool valid, int32_t r, int32_t a, int32_t lp)
    {
        const int32_t a2 = a2base + (lp - lpbase);
        int32_t x0 = 0, y0 = 0;
        uint32_t c = 0;
        if (valid) c = pair_xy<TAB>(q, X0, YD, r, x0, y0);
        if (__any_sync(FULL, c > (uint32_t)ENUM_BIG)) {
            // rare: a leaf with very many rows; one leaf at a time
            for (int src = 0; src < 32; src++) {
                const uint32_t cs = __shfl_sync(FULL, c, src);
                if (cs == 0) continue;
                const bool me = lane == src;
                emit(q, lane, cs, me ? 0u : cs, cs, x0, y0, a, a2);
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
        if (T > 0) emit(q, lane, T, incl - c, incl, x0, y0, a, a2);
        return false;
    }
};

template <bool TAB, typename ELEM, int MAXL>
__global__ void __launch_bounds__(256, 3) k_pair_enum(const __grid_constant__ QueryConst q,
                                                      Scratch sc, int queue, ELEM* out,
                                                      uint64_t cap_rows)
{
    __shared__ SmemQ sq;
    extern __shared__ __align__(16) unsigned char dyn[];
    load_smemq(q, sq, sc.ctr);
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
    using C = EnumCons<TAB, ELEM, MAXL>;
    C cons;
    cons.sg.out = out;
    cons.sg.cap_elems = cap_rows * (uint64_t)q.d;
    cons.sg.lo_elems = sc.row_lo * (uint64_t)q.d;
    cons.sg.wbase = wp;
    cons.sg.d = q.d;
    cons.sg.begin(0);
    cons.X0 = X0;
    cons.YD = YD;
    cons.slice_off = sc.slice_off;
    cons.blk = sc.blk;
    cons.map = wp + ENUM_STG_BYTES;
    cons.tmpl = (int32_t*)(wp + ENUM_STG_BYTES + ENUM_MAPCAP);
    cons.scol = sq.col;
    cons.ctr = sc.ctr;
    cons.np = q.P - 1;
    const int piece = (Stager<ELEM>::STG - Stager<ELEM>::VEC) / q.d;
    cons.piece = piece < ENUM_MAPCAP ? piece : ENUM_MAPCAP;
    cons.cin = q.col[q.P - 1];
    cons.cA = q.col[q.P];
    cons.cB = q.col[q.P + 1];
#pragma unroll
    for (int k = 0; k < C::NR; k++) {
        cons.col[k] = q.col[k];
        cons.pre[k] = 0;
    }
    run_queue(q, sq, sc, queue, cons);
    cons.sg.finish();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int pair_enum_smem_bytes(const QueryConst& q, int threads, int)
{
    const int tab = q.tab_xy ? (((int)q.lcm * 8 + 15) & ~15) : 0;
    return tab + (threads / 32) * ENUM_WARP_BYTES;
}

template <bool TAB, typename ELEM>
static void* pick(const QueryConst& q)
{
    if (q.D <= 4) return (void*)k_pair_enum<TAB, ELEM, 4>;
    if (q.D <= 8) return (void*)k_pair_enum<TAB, ELEM, 8>;
    return (void*)k_pair_enum<TAB, ELEM, 16>;
}

static void* enum_kernel(const QueryConst& q, int elem_bytes)
{
    if (void* k = pair_enum_fixed_kernel(q, elem_bytes)) return k;
    if (elem_bytes == 2) return q.tab_xy ? pick<true, int16_t>(q) : pick<false, int16_t>(q);
    return q.tab_xy ? pick<true, int32_t>(q) : pick<false, int32_t>(q);
}

cudaError_t pair_enum_occupancy(const QueryConst& q, int threads, int elem_bytes, int* nb)
{
    const void* k = enum_kernel(q, elem_bytes);
    const int smem = pair_enum_smem_bytes(q, threads, elem_bytes);
    return occupancy_cached(k, threads, smem, nb);
}

cudaError_t launch_pair_enum(const QueryConst& q, const Scratch& sc, const LaunchCfg& lc, int queue,
                             void* out, uint64_t cap_rows, int elem_bytes, cudaStream_t st)
{
    const void* k = enum_kernel(q, elem_bytes);
    const int smem = pair_enum_smem_bytes(q, lc.threads, elem_bytes);
    cudaError_t e = smem_optin(k, smem);
    if (e != cudaSuccess) return e;
    QueryConst qq = q;
    Scratch ss = sc;
    int qu = queue;
    uint64_t cr = cap_rows;
    void* args[] = {&qq, &ss, &qu, &out, &cr};
    return cudaLaunchKernel(k, dim3(lc.blocks), dim3(lc.threads), args, (size_t)smem, st);
}

}  // namespace fsi
