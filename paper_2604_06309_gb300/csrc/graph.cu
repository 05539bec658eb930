// Step graphs. A Dormand-Prince step has 6 stage evaluations, an SSPRK(10,4) step 10
// (Sec. 3.5). One graph serves both: the first 6 stages are plain nodes, the last 4 sit
// in the body of a conditional IF node whose condition the step's first kernel sets from
// the device-side method word, so Dormand-Prince steps launch no idle stage kernels and
// the host never has to know which method the device chose.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "dmfe_internal.h"

// DMFE_STEP_GRAPH=plain selects step graphs without the conditional node (all stages
// inline, the SSPRK ones gating themselves off): profilers that cannot attribute kernels
// inside graphs with conditional nodes then see every kernel of a step.
bool step_graph_plain() {
    const char* e = std::getenv("DMFE_STEP_GRAPH");
    return e && std::strcmp(e, "plain") == 0;
}

namespace {

int capture_plain(cudaStream_t cap, StepParts& parts, cudaGraph_t* g) {
    DMFE_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int rc = parts.head(0, 0, cap);
    if (!rc) rc = parts.tail(cap);
    if (!rc) rc = parts.sp(cap);
    const cudaError_t e = cudaStreamEndCapture(cap, g);
    if (rc || e != cudaSuccess) {
        if (*g) cudaGraphDestroy(*g);
        *g = nullptr;
        cudaGetLastError();
        return rc ? rc : DMFE_ERR_CUDA;
    }
    return DMFE_OK;
}

int capture_conditional(cudaStream_t cap, StepParts& parts, cudaGraph_t* g) {
    cudaStream_t body_stream = nullptr;
    DMFE_CUDA_TRY(cudaStreamCreateWithFlags(&body_stream, cudaStreamNonBlocking));
    int rc = DMFE_OK;
    bool capturing = false;
    do {
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = DMFE_ERR_CUDA; break; }
        capturing = true;
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        if (cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess ||
            cs != cudaStreamCaptureStatusActive) { rc = DMFE_ERR_CUDA; break; }
        cudaGraphConditionalHandle cond = 0;
        // default 0 at every launch: the body runs only when the first kernel sets 1
        if (cudaGraphConditionalHandleCreate(&cond, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
            rc = DMFE_ERR_CUDA;
            break;
        }
        rc = parts.head(cond, 1, cap);
        if (rc) break;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if (cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess) {
            rc = DMFE_ERR_CUDA;
            break;
        }
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np) != cudaSuccess) { rc = DMFE_ERR_CUDA; break; }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = DMFE_ERR_CUDA;
            break;
        }
        rc = parts.tail(body_stream);
        cudaGraph_t body_out = nullptr;
        const cudaError_t eb = cudaStreamEndCapture(body_stream, &body_out);
        if (rc || eb != cudaSuccess) { rc = rc ? rc : DMFE_ERR_CUDA; break; }
        if (cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
            cudaSuccess) {
            rc = DMFE_ERR_CUDA;
            break;
        }
        rc = parts.sp(cap);
    } while (false);
    if (capturing) {
        cudaGraph_t gg = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &gg);
        if (rc || e != cudaSuccess) {
            if (gg) cudaGraphDestroy(gg);
            rc = rc ? rc : DMFE_ERR_CUDA;
        } else {
            *g = gg;
        }
    }
    cudaStreamDestroy(body_stream);
    if (rc) cudaGetLastError();
    return rc;
}

}  // namespace

int capture_step_graph(cudaStream_t cap, bool conditional, StepParts& parts, cudaGraphExec_t* out) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    int rc = conditional ? capture_conditional(cap, parts, &g) : capture_plain(cap, parts, &g);
    if (rc) return rc;
    const cudaError_t e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        cudaGetLastError();
        return DMFE_ERR_CUDA;
    }
    return DMFE_OK;
}
