// CUDA-graph replay of a pair's launch sequence. One capture per combination of caller
// pointers and pyramid slots; later calls with the same combination replay it, so a
// stream of frames on fixed buffers costs one graph launch per field.
#include "of_engine.h"
#include "of_internal.cuh"

namespace of {

void drop_graphs(of_ctx *h)
{
    for (int i = 0; i < h->n_graphs; ++i)
        if (h->graphs[i].exec) cudaGraphExecDestroy(h->graphs[i].exec);
    h->n_graphs = 0;
}

static int capture(of_ctx *h, const void *I1, const void *I2, float *u, float *v, int s1, int s2, cudaStream_t st,
                   cudaGraph_t *g)
{
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return OF_ECUDA;
    cudaError_t le = enqueue_pair(h, I1, I2, u, v, s1, s2, st);
    e = cudaStreamEndCapture(st, g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (*g) cudaGraphDestroy(*g);
        *g = nullptr;
        cudaGetLastError();
        return OF_ECUDA;
    }
    return OF_OK;
}

int run_pair(of_ctx *h, const void *I1, const void *I2, float *u, float *v, int s1, int s2, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool graphs = st != nullptr && !(h->plan.flags & OF_FLAG_NO_GRAPH) &&
                        cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    if (!graphs) return enqueue_pair(h, I1, I2, u, v, s1, s2, st) == cudaSuccess ? OF_OK : OF_ECUDA;

    ++h->use_clock;
    for (int i = 0; i < h->n_graphs; ++i) {
        GraphEntry &g = h->graphs[i];
        if (g.I1 == I1 && g.I2 == I2 && g.u == u && g.v == v && g.s1 == s1 && g.s2 == s2) {
            g.last_use = h->use_clock;
            return cudaGraphLaunch(g.exec, st) == cudaSuccess ? OF_OK : OF_ECUDA;
        }
    }
    cudaGraph_t graph = nullptr;
    int rc = capture(h, I1, I2, u, v, s1, s2, st, &graph);
    if (rc) return rc;
    // reuse the least recently used slot when the cache is full
    int slot = h->n_graphs;
    if (slot == GRAPH_CACHE) {
        slot = 0;
        for (int i = 1; i < GRAPH_CACHE; ++i)
            if (h->graphs[i].last_use < h->graphs[slot].last_use) slot = i;
    }
    GraphEntry &g = h->graphs[slot];
    bool ok = false;
    if (slot < h->n_graphs && g.exec) {
        cudaGraphExecUpdateResultInfo info;
        ok = cudaGraphExecUpdate(g.exec, graph, &info) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
    }
    if (!ok) {
        if (cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            g.exec = nullptr;
            if (slot < h->n_graphs) {   // drop the emptied slot
                h->graphs[slot] = h->graphs[h->n_graphs - 1];
                --h->n_graphs;
            }
            return OF_ECUDA;
        }
    }
    cudaGraphDestroy(graph);
    if (slot == h->n_graphs) ++h->n_graphs;
    g.I1 = I1;
    g.I2 = I2;
    g.u = u;
    g.v = v;
    g.s1 = s1;
    g.s2 = s2;
    g.last_use = h->use_clock;
    return cudaGraphLaunch(g.exec, st) == cudaSuccess ? OF_OK : OF_ECUDA;
}

}  // namespace of
