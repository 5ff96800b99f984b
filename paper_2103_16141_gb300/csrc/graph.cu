// Device-side Lloyd loop (Algorithm 1) for use_graph contexts: one CUDA graph
// whose conditional WHILE node repeats [assignment, update, loop control]
// until every instance has converged or the iteration cap is reached. The
// control kernel decides on the device, so iterations run back to back with
// no host round trip; the host launches the graph once per sivf_run call.
#include "sivf_internal.cuh"

namespace sivf {
namespace {

// loop[0] = r of the last assignment, loop[1] = iteration cap, loop[2] = instances
// still running. An instance converges at the first assignment r > 1 that changes
// none of its labels (done[m] = r); until then objf[m] follows its update objective.
__global__ void loop_control(cudaGraphConditionalHandle h, int32_t *loop, int32_t n_inst,
                             const unsigned long long *inst_changed, const DevCounters *ctr, const double *obj,
                             int32_t *done, double *objf) {
    __shared__ int rem;
    if (threadIdx.x == 0) rem = 0;
    __syncthreads();
    const int r = loop[0] + 1;
    for (int m = threadIdx.x; m < n_inst; m += blockDim.x) {
        const unsigned long long ch = n_inst == 1 ? ctr->changed : inst_changed[m];
        if (done[m] == 0) {
            if (r > 1 && ch == 0) {
                done[m] = r;
            } else {
                objf[m] = obj[2 * m + 1];
                atomicAdd(&rem, 1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        loop[0] = r;
        loop[2] = rem;
        cudaGraphSetConditional(h, (rem > 0 && r < loop[1]) ? 1u : 0u);
    }
}

}  // namespace

void destroy_loop_graph(sivf_ctx *c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
}

cudaError_t build_loop_graph(sivf_ctx *c) {
    destroy_loop_graph(c);
    cudaGraph_t g = nullptr;
    SIVF_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // capture on a private stream: the caller's stream may be the legacy
    // default stream, which cannot be captured; the graph is launched on the
    // caller's stream afterwards
    cudaStream_t user = c->stream, cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        cudaGraphDestroy(g);
        c->err = "begin capture failed";
        return e;
    }
    c->stream = cap;
    const unsigned long long l0 = g_launches;
    cudaError_t e1 = enqueue_assign(c, false);
    cudaError_t e2 = e1 == cudaSuccess ? enqueue_update(c, false) : cudaSuccess;
    if (e1 == cudaSuccess && e2 == cudaSuccess) {
        loop_control<<<1, 256, 0, cap>>>(h, c->loop_dev, c->n_inst, c->inst_changed, c->ctr, c->obj_dev,
                                               c->done_dev, c->objf_dev);
        note_launch();
    }
    c->launches_per_iter = g_launches - l0;
    cudaGraph_t captured = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(cap, &captured);
    cudaError_t e4 = cudaGetLastError();
    c->stream = user;
    cudaStreamDestroy(cap);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
        cudaGraphDestroy(g);
        c->err = e1 != cudaSuccess ? "capture of the assignment step failed"
                 : e2 != cudaSuccess ? "capture of the update step failed"
                                     : "end of capture failed";
        return e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    c->graph = g;
    c->graph_exec = exec;
    return cudaSuccess;
}

}  // namespace sivf
