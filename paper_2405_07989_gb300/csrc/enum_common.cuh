// Shared pieces of the enumerate write walks (enum.cu, enum_fixed.cu): the
// bulk-copy helpers and the per-warp staging of rows.
#pragma once

#include "walk.cuh"

namespace fsi {

enum { ENUM_STG_BYTES = 6144, ENUM_MAPCAP = 256, ENUM_BIG = 1 << 26 };
// per warp: the staging buffer, the row -> lane map, the run prefix of the
// generic (d > 8) path
enum { ENUM_WARP_BYTES = ENUM_STG_BYTES + ENUM_MAPCAP + 2 * FS_MAX_D * 4 };

// --- bulk async copies, shared -> global (PTX cp.async.bulk, bulk groups) ---
FS_D void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

FS_D void bulk_store(void* gdst, const void* ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                     (unsigned long long)__cvta_generic_to_global(gdst)),
                 "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes)
                 : "memory");
}
FS_D void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every group has read its shared memory (the source may be rewritten)
FS_D void bulk_wait_read_0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every group complete (writes performed)
FS_D void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Per-warp staging of consecutive output rows in shared memory, drained by
// the bulk-copy engine.  The staged rows are the global rows
// [row_base, row_base + nst); global element g (= row * d + column) goes to
// out[g - lo_elems] when 0 <= g - lo_elems < cap_elems and is dropped
// otherwise (the window of a cursor; lo_elems = 0 for a whole enumerate).
// Staged element e sits at index phase + e of the current buffer, with
// phase = (row_base d - lo_elems) mod VEC so that 16-byte boundaries line up
// with the output's.
template <typename ELEM>
struct Stager {
    static constexpr int VEC = 16 / (int)sizeof(ELEM);
    static constexpr int STG = ENUM_STG_BYTES / (int)sizeof(ELEM);
    ELEM* out;
    uint64_t cap_elems;
    uint64_t lo_elems;
    unsigned char* wbase;  // this warp's staging buffer
    uint64_t row_base;
    int32_t nst, phase, d;

    FS_D ELEM* stg() const { return (ELEM*)wbase; }
    FS_D ELEM* cursor() const { return stg() + phase + nst * d; }
    FS_D bool fits(int rows) const { return phase + (nst + rows) * d <= STG; }
    // rows that still fit the buffer (D: the row width, d, as a constant)
    template <int D>
    FS_D uint32_t room() const { return (uint32_t)((STG - phase) / D - nst); }
    // window position of the first staged element (negative: before the window)
    FS_D int64_t wpos() const { return (int64_t)(row_base * (uint64_t)d) - (int64_t)lo_elems; }

    FS_D void begin(uint64_t row0)
    {
        row_base = row0;
        nst = 0;
        phase = (int32_t)(((wpos() % VEC) + VEC) % VEC);
    }

    // Write the staged rows that fall in the window and switch buffers.
    FS_D void flush()
    {
        const int lane = threadIdx.x & 31;
        __syncwarp();  // every lane's staged rows are in place
        if (nst > 0) {
            const ELEM* sb = stg();
            const int64_t e0 = wpos();
            const int64_t N = (int64_t)nst * d;
            const int64_t lo = e0 > 0 ? e0 : 0;
            const int64_t hi = (e0 + N < (int64_t)cap_elems) ? e0 + N : (int64_t)cap_elems;
            if (lo < hi) {
                // staged index of window element e: phase + (e - e0)
                const int32_t sb0 = phase + (int32_t)(lo - e0);
                const uint64_t g0 = (uint64_t)lo;
                const uint32_t span = (uint32_t)(hi - lo);
                uint32_t head = (uint32_t)((VEC - g0 % VEC) % VEC);
                if (head > span) head = span;
                const uint32_t nv = (span - head) / VEC;
                const uint32_t tail0 = head + nv * VEC;
                if ((uint32_t)lane < head) out[g0 + lane] = sb[sb0 + lane];
                for (uint32_t i = tail0 + lane; i < span; i += 32) out[g0 + i] = sb[sb0 + i];
                if (nv > 0) {
                    fence_proxy_async_smem();  // staging writes -> visible to the bulk copy
                    __syncwarp();
                    if (lane == 0) {
                        bulk_store(out + g0 + head, sb + sb0 + head, nv * 16u);
                        bulk_commit();
                    }
                }
            }
            // one buffer per warp, reused at once: its copy must have read it.
            // (Two half-size buffers, one filling while the other drains,
            // flush twice as often and measured slower.)
            if (lane == 0) bulk_wait_read_0();
            __syncwarp();
        }
        row_base += (uint64_t)nst;
        nst = 0;
        phase = (int32_t)(((wpos() % VEC) + VEC) % VEC);
    }

    FS_D void finish()
    {
        if ((threadIdx.x & 31) == 0) bulk_wait_all();
        __syncwarp();
    }
};

}  // namespace fsi
