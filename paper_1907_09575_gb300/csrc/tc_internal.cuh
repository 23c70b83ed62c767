// Declarations shared between the preprocessing, counting and API units.
#pragma once
#include "common.cuh"

namespace tc {

constexpr int kSmallTable = 128;     // hash slots of a warp unit's table
constexpr int kSmallMaxOutdeg = 64;  // largest pivot row a warp unit takes
constexpr int kMaxSlice = 4096;      // largest pivot slice a CTA unit tables
constexpr int kMaxUnitTasks = 8192;  // 16-bit hit counters; a shared long-task queue

void tuning_defaults(tc_tuning* t);
void tuning_resolve(const tc_tuning* in, tc_tuning* out);  // fills zeros, clamps
bool tuning_equal(const tc_tuning& a, const tc_tuning& b);

void preprocess(tc_graph* g, const int32_t* src, const int32_t* dst, int64_t P, uint32_t flags,
                cudaStream_t st);
void build_units(tc_graph* g, const tc_tuning& t, cudaStream_t st);
void count(const tc_graph* g, const tc_tuning& t, uint64_t* total_dev, uint64_t* per_vertex_dev,
           cudaStream_t st);

}  // namespace tc
