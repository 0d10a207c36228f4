// flood_graph.cpp -- whole CFL epochs (epoch start, Eq. 6 inflow, E step
// launches) captured once into a CUDA graph and replayed, which removes the
// per-launch CPU cost that dominates small grids.  Two graphs exist, one per
// parity of the ping-pong buffer at the epoch start.
#include "flood_runtime.h"

namespace flood {

static flood_status capture_epoch(flood_handle *h, int parity)
{
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "capture stream");
    cudaStream_t user = h->stream;
    const int64_t step0 = h->step;
    const int cur0 = h->cur;
    h->stream = cap;
    h->cur = parity;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    flood_status st = FLOOD_OK;
    if (e == cudaSuccess) st = advance(h, h->geo.epoch_steps, nullptr, 0, nullptr, nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    h->stream = user;
    h->step = step0;
    h->cur = cur0;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "end capture");
    e = cudaGraphInstantiate(&h->graph_exec[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph_exec[parity] = nullptr;
        return cuda_fail(h, e, "graph instantiate");
    }
    return FLOOD_OK;
}

flood_status advance_graph(flood_handle *h, int64_t n)
{
    const int E = h->geo.epoch_steps;
    while (n > 0) {
        int s = (int)(h->step % E);
        if (s != 0 || n < E) {
            int64_t k = s != 0 ? std::min<int64_t>(E - s, n) : n;
            flood_status st = advance(h, k, nullptr, 0, nullptr, nullptr);
            if (st) return st;
            n -= k;
            continue;
        }
        int parity = h->cur;
        if (!h->graph_exec[parity]) {
            flood_status st = capture_epoch(h, parity);
            if (st) return st;
        }
        cudaError_t e = cudaGraphLaunch(h->graph_exec[parity], h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
        h->step += E;
        h->cur = (h->cur + (h->kernel == FLOOD_KERNEL_TILED ? E / h->k_per_launch : E)) & 1;
        n -= E;
    }
    return FLOOD_OK;
}

void invalidate_graphs(flood_handle *h)
{
    for (int p = 0; p < 2; p++)
        if (h->graph_exec[p]) {
            cudaGraphExecDestroy(h->graph_exec[p]);
            h->graph_exec[p] = nullptr;
        }
}

void destroy_graphs(flood_handle *h) { invalidate_graphs(h); }

}  // namespace flood
