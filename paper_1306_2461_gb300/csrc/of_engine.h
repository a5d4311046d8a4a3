// Host-side engine state of libof: the handle, its workspace layout, graph cache.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/of.h"

namespace of {

constexpr int MAX_LEVELS = 16;
constexpr int GRAPH_CACHE = 4;

struct Layout {
    int levels;
    int H[MAX_LEVELS], W[MAX_LEVELS], pitch[MAX_LEVELS];
    size_t level_off[MAX_LEVELS];   // byte offset of each level inside a pyramid slot
    size_t pyr_bytes;               // one pyramid slot
    size_t flow_bytes;              // one float2 flow buffer (level 0, pitched)
    size_t hess_off, hess_bytes;    // window matrices of the first-image-gradient variant (0 bytes otherwise)
    size_t total;
};

// A replayable launch sequence for one combination of caller pointers and slots.
struct GraphEntry {
    const void *I1, *I2;
    float *u, *v;
    int s1, s2;
    cudaGraphExec_t exec;
    uint64_t last_use;
};

void layout_plan(const of_plan &p, Layout &L);

}  // namespace of

struct of_ctx {
    of_plan plan;
    of::Layout lay;
    int device = 0;
    char *ws = nullptr;              // the one workspace allocation
    char *pyr[2] = {nullptr, nullptr};
    float2 *flow[2] = {nullptr, nullptr};
    int *status = nullptr;           // device status word
    float4 *hess = nullptr;          // OF_FLAG_I1GRAD: (Sa, Sb, Sc, 0) of the level being iterated
    cudaEvent_t done = nullptr;      // recorded after each compute
    cudaStream_t ctl = nullptr;      // private stream for status reads
    bool has_prev = false;           // a previous second image's pyramid is resident
    int prev_slot = 1;
    int last_s1 = 0, last_s2 = 1;
    bool computed = false;
    of::GraphEntry graphs[of::GRAPH_CACHE] = {};
    int n_graphs = 0;
    uint64_t use_clock = 0;
};

namespace of {

// Point the handle's buffers into a workspace of lay.total bytes laid out by layout_plan.
void assign_workspace(of_ctx *h, char *ws);
cudaError_t enqueue_pair(of_ctx *h, const void *I1, const void *I2, float *u, float *v, int s1, int s2,
                         cudaStream_t st);
// Queue one pair through a cached CUDA graph when the stream allows it, else directly.
int run_pair(of_ctx *h, const void *I1, const void *I2, float *u, float *v, int s1, int s2, cudaStream_t st);
void drop_graphs(of_ctx *h);

// A reusable launch slot for the persistent batch kernel: device and pinned host
// buffers for the descriptors of up to max_pairs pairs and max_phases phases.
// cudaMalloc that honours of_debug_fail_allocs (injected out-of-memory failures).
cudaError_t dev_malloc(void **p, size_t bytes);

// How one persistent batched launch is run (the autotuner's choice; see tune.cu).
struct Tuning {
    int generic_sums = 0;    // 1: the run-time-radius kernel (per-output sums); 0: grouped fixed-radius sums
    int stage_i2 = 1;        // 1: stage I2 windows and estimates in shared memory (fixed-radius kernel only)
    int blocks_per_sm = 0;   // resident blocks per SM of the persistent launch; 0 = as many as fit
    int phased = 1;          // 1: one ordinary launch per phase; 0: the persistent launch with grid barriers
    int prefetch = 0;        // phase launches: warm L2 for the tile this many blocks per SM ahead (0: off)
    int tile_h = 0;          // phase launches with grouped sums: iteration tile height (0: the default)
    int branches = 0;        // phase launches: concurrent launch sequences over parts of the batch (0: one)
    int fusion = 0;          // phase launches: 2 fuses pairs of same-level iterations in one launch per tile
                             // (fixed radii, default tile height); 0 or 1: one iteration per launch
    int strip = 0;           // phase launches with grouped sums: tiles per block along y (1, 2, 4; 0: 4)
};
// Tiles per block along y of a tuning's phase launches of grouped sums.
inline int tuning_strip(const Tuning &t) { return t.strip ? t.strip : 4; }
// The tuning table entry for this method and size class, or the default.
Tuning tuning_for(const of_plan &method, int size_class);
// round(log2(mean level-0 pixels per pair)) of a batch.
int batch_size_class(int32_t n, const of_handle *hs);
int run_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s, float *const *us,
              float *const *vs, cudaStream_t st, const Tuning &t);
// Whether two plans can share a batched launch (same method; sizes may differ).
bool same_method(const of_plan &a, const of_plan &b);

struct BatchSlot {
    char *dev = nullptr;
    char *host = nullptr;
    size_t desc_bytes = 0;
    int max_pairs = 0, max_phases = 0;
    cudaEvent_t done = nullptr;
};
int batch_slot_init(BatchSlot &s, int max_pairs, int max_phases);
void batch_slot_free(BatchSlot &s);
int batch_run_slot(BatchSlot &slot, int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                   float *const *us, float *const *vs, cudaStream_t st);

}  // namespace of
