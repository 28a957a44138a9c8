// Host-side launchers implemented in the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include "fs_internal.h"

namespace fsi {

// Launch attributes asked of the runtime once per device / kernel / shape
// (hostcache.cu): blocks per SM, the dynamic shared-memory opt-in, the SM
// count.
cudaError_t occupancy_cached(const void* kern, int threads, int smem, int* nb);
cudaError_t smem_optin(const void* kern, int smem);
cudaError_t sm_count_cached(int* sms);

// Every device and pinned-host allocation of the library goes through these
// (hostcache.cu), which count the successful ones (fs_alloc_counts).
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t host_alloc(void** p, size_t bytes);


enum Op { OP_COUNT = 0, OP_SLICES = 1, OP_LEN = 2, OP_ANY = 3, OP_ENUM = 4 };

struct LaunchCfg {
    int threads;
    int blocks;
    uint64_t S;           // slices (the maximum, when auto_s)
    int auto_s;           // 1: the planner picks min(S, ceil(L / min_leaves)) slices;
                          // 2: the same with a tail of short slices (make_split)
    uint64_t min_leaves;
};

// tables.cu
// The walk query's tables (leaf counts, pair tables) and, with qt and
// trail_k > 0, the trailing-k tables of qt (T, and MN / MX when not NULL):
// one launch, one block per table.
cudaError_t launch_precompute(const QueryConst& q, const Scratch& sc, cudaStream_t st,
                              const QueryConst* qt = nullptr, int trail_k = 0, uint64_t* T = nullptr,
                              int32_t* MN = nullptr, int32_t* MX = nullptr);
cudaError_t launch_scan_slices(const Scratch& sc, uint64_t* dev_count, cudaStream_t st);
cudaError_t launch_len_finalize(const QueryConst& q, const Scratch& sc, uint64_t* hist, int s,
                                cudaStream_t st);
cudaError_t launch_copy_u64(const uint64_t* src, uint64_t* dst, cudaStream_t st);
cudaError_t launch_len_summary(const Scratch& sc, uint64_t* out, cudaStream_t st);

// pair.cu  (closed-form pair, warp-cooperative walk)
int pair_smem_bytes(const QueryConst& q, Op op, int threads, int elem_bytes);
cudaError_t pair_occupancy(const QueryConst& q, Op op, int threads, int elem_bytes, int* blocks_per_sm);
cudaError_t launch_pair(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                        int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                        int elem_bytes, cudaStream_t st);

// pair.cu: the TRIPLE walk over the reduced query q3 (OP_COUNT, OP_SLICES,
// OP_LEN = count + min / max length)
// The trailing-table walk: its block size for q3 / op, and blocks per SM.
int triple_threads(const QueryConst& q3, Op op);
// Kernels launch_triple enqueues for op (2 for a length range in shared memory).
int triple_walk_kernels(const QueryConst& q3, Op op);
cudaError_t triple_occupancy(const QueryConst& q3, Op op, int threads, int* blocks_per_sm);
// Enumerate's first walk, run by run (k_pair_slice_runs): per-slice counts,
// the two-level offsets of Scratch::blk, the total (ctr[CTR_TOTAL] and, if
// not NULL, *dev_count).  S_req: the planner's maximum slice count.
// The planner and enumerate's slice offsets in one launch, from prefix-count
// tables in shared memory (k_plan_offsets); usable when plan_runs_smem_bytes(q)
// fits.  Offsets are global (Scratch::blk unused).
size_t plan_runs_smem_bytes(const QueryConst& q);
cudaError_t launch_plan_runs(const QueryConst& q, const Scratch& sc, uint64_t S_req, int auto_s,
                             uint64_t min_leaves, uint64_t* dev_count, cudaStream_t st);
cudaError_t launch_pair_slice_runs(const QueryConst& q, const Scratch& sc, const uint64_t* T3,
                                   uint64_t S_req, uint64_t* dev_count, cudaStream_t st);
cudaError_t launch_triple(const QueryConst& q3, const Scratch& sc, Op op, const LaunchCfg& lc,
                          int queue, const uint64_t* T3, const int32_t* MN3, const int32_t* MX3,
                          uint64_t* dev_count, cudaStream_t st);

// enum_fixed.cu: the write walk specialised on the number of levels and a
// caller-order / reversed column order; NULL when the query has neither.
void* pair_enum_fixed_kernel(const QueryConst& q, int elem_bytes);

// enum.cu  (closed-form pair, enumerate write walk)
int pair_enum_smem_bytes(const QueryConst& q, int threads, int elem_bytes);
cudaError_t pair_enum_occupancy(const QueryConst& q, int threads, int elem_bytes, int* blocks_per_sm);
cudaError_t launch_pair_enum(const QueryConst& q, const Scratch& sc, const LaunchCfg& lc, int queue,
                             void* out, uint64_t cap_rows, int elem_bytes, cudaStream_t st);

// plain.cu  (Algorithm 3.1 per thread)
cudaError_t plain_occupancy(const QueryConst& q, Op op, int threads, int* blocks_per_sm);
cudaError_t launch_plain(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                         int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                         int elem_bytes, cudaStream_t st);

// batch.cu
cudaError_t batch_walk_occupancy(int mode, int threads, int* blocks_per_sm);
cudaError_t launch_batch(const BatchDev& b, int threads, int blocks, cudaStream_t st);

// probe.cu: integer throughput of kind 0 (add), 1 (lop3), 2 (mad) on the whole GPU
cudaError_t int_probe(int kind, uint32_t iters, double* ops_per_s, double* ms_out);

// tables.cu: the slice planner.  S_req slices, or with auto_s the number of
// slices min(S_req, ceil(L / min_leaves)) (at least 1), written to ctr[CTR_SEFF]
// together with L (ctr[CTR_L]) and every slice's start state (sc.starts).
cudaError_t launch_plan(const QueryConst& q, const Scratch& sc, uint64_t S_req, int auto_s,
                        uint64_t min_leaves, cudaStream_t st);

}  // namespace fsi
