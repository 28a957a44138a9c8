// Host-side launchers implemented in the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include "fs_internal.h"

namespace fsi {

enum Op { OP_COUNT = 0, OP_SLICES = 1, OP_LEN = 2, OP_ANY = 3, OP_ENUM = 4 };

struct LaunchCfg {
    int threads;
    int blocks;
    uint64_t S;  // slices
};

// tables.cu
cudaError_t launch_precompute(const QueryConst& q, const Scratch& sc, cudaStream_t st);
cudaError_t launch_scan_slices(const Scratch& sc, uint64_t S, uint64_t* dev_count, cudaStream_t st);
cudaError_t launch_len_finalize(const QueryConst& q, const Scratch& sc, uint64_t* hist, int s,
                                cudaStream_t st);
cudaError_t launch_copy_u64(const uint64_t* src, uint64_t* dst, cudaStream_t st);

// pair.cu  (closed-form pair, warp-cooperative walk)
int pair_smem_bytes(const QueryConst& q, Op op, int threads, int elem_bytes);
cudaError_t pair_occupancy(const QueryConst& q, Op op, int threads, int elem_bytes, int* blocks_per_sm);
cudaError_t launch_pair(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                        int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                        int elem_bytes, cudaStream_t st);

// plain.cu  (Algorithm 3.1 per thread)
cudaError_t plain_occupancy(const QueryConst& q, Op op, int threads, int* blocks_per_sm);
cudaError_t launch_plain(const QueryConst& q, const Scratch& sc, Op op, const LaunchCfg& lc,
                         int queue, const PredConst* pred, void* out, uint64_t cap_rows,
                         int elem_bytes, cudaStream_t st);

// plan.cu
cudaError_t launch_plan_bounds(const QueryConst& q, const Scratch& sc, uint64_t S, int32_t* bounds,
                               cudaStream_t st);

}  // namespace fsi
