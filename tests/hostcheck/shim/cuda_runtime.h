// Test double of the CUDA runtime surface that plan.cpp uses, so that the
// planner and sweep driver can be exercised on a CPU-only host with host memory.
// TEST INFRASTRUCTURE ONLY: never part of the product library.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <vector>

typedef int cudaError_t;
typedef void* cudaStream_t;
enum { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorNotSupported = 801,
       cudaErrorMemoryAllocation = 2 };
enum cudaMemcpyKind { cudaMemcpyHostToDevice = 1, cudaMemcpyDeviceToHost = 2,
                      cudaMemcpyDeviceToDevice = 3 };

inline cudaError_t cudaMalloc(void** p, size_t n) {
    *p = std::malloc(n ? n : 1);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
template <typename T>
inline cudaError_t cudaMalloc(T** p, size_t n) {
    return cudaMalloc(reinterpret_cast<void**>(p), n);
}
inline cudaError_t cudaFree(void* p) { std::free(p); return cudaSuccess; }
inline cudaError_t cudaMemset(void* p, int v, size_t n) { std::memset(p, v, n); return cudaSuccess; }
// Stream capture: while a capture is open, launches and async copies are
// recorded instead of run; a graph launch replays them in order.
// Captures nest (a conditional node's body is captured while its parent graph's
// capture is open): the innermost open capture receives the work.  A while node
// is one operation of its graph that runs the body's operations while its
// condition value (set by the mock kernels) is nonzero.
struct HostGraph {
    std::vector<std::function<void()>> ops;  // a while node's operation shares its body
};
typedef HostGraph* cudaGraph_t;
typedef HostGraph* cudaGraphExec_t;
inline std::vector<HostGraph*>& host_captures() {
    static std::vector<HostGraph*> g;
    return g;
}
inline HostGraph* host_capture() { return host_captures().empty() ? nullptr : host_captures().back(); }
template <class F>
inline cudaError_t host_submit(F f) {
    if (host_capture()) {
        host_capture()->ops.push_back([f]() { (void)f(); });
        return cudaSuccess;
    }
    return f();
}
enum cudaStreamCaptureMode { cudaStreamCaptureModeGlobal = 0, cudaStreamCaptureModeThreadLocal = 1,
                             cudaStreamCaptureModeRelaxed = 2 };
enum { cudaStreamNonBlocking = 1, cudaEventDisableTiming = 2 };
inline cudaError_t cudaStreamBeginCapture(cudaStream_t, cudaStreamCaptureMode) {
    host_captures().push_back(new HostGraph);
    return cudaSuccess;
}
inline cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t* g) {
    HostGraph* top = host_captures().back();
    host_captures().pop_back();
    if (g) *g = top;
    return cudaSuccess;
}
typedef unsigned long long cudaGraphConditionalHandle;
typedef struct HostNode* cudaGraphNode_t;
struct cudaGraphEdgeData;
enum cudaStreamCaptureStatus { cudaStreamCaptureStatusNone = 0, cudaStreamCaptureStatusActive = 1 };
enum { cudaStreamAddCaptureDependencies = 0, cudaStreamSetCaptureDependencies = 1 };
enum { cudaGraphCondAssignDefault = 1 };
enum cudaGraphConditionalNodeType { cudaGraphCondTypeIf = 0, cudaGraphCondTypeWhile = 1 };
enum cudaGraphNodeType { cudaGraphNodeTypeKernel = 0, cudaGraphNodeTypeConditional = 0x0d };
struct cudaConditionalNodeParams {
    cudaGraphConditionalHandle handle;
    cudaGraphConditionalNodeType type;
    unsigned int size;
    cudaGraph_t* phGraph_out;
};
struct cudaGraphNodeParams {
    cudaGraphNodeType type;
    cudaConditionalNodeParams conditional;
};
inline cudaError_t cudaStreamGetCaptureInfo(cudaStream_t, cudaStreamCaptureStatus* status, unsigned long long*,
                                            cudaGraph_t* graph, const cudaGraphNode_t** deps,
                                            const cudaGraphEdgeData**, size_t* n_deps) {
    if (status) *status = host_capture() ? cudaStreamCaptureStatusActive : cudaStreamCaptureStatusNone;
    if (graph) *graph = host_capture();
    if (deps) *deps = nullptr;
    if (n_deps) *n_deps = 0;
    return cudaSuccess;
}
// a handle is the address of its condition value
inline cudaError_t cudaGraphConditionalHandleCreate(cudaGraphConditionalHandle* h, cudaGraph_t, unsigned def,
                                                    unsigned) {
    static std::vector<unsigned*> values;
    values.push_back(new unsigned(def));
    *h = reinterpret_cast<cudaGraphConditionalHandle>(values.back());
    return cudaSuccess;
}
inline cudaError_t cudaGraphAddNode(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t*,
                                    const cudaGraphEdgeData*, size_t, cudaGraphNodeParams* np) {
    if (np->type != cudaGraphNodeTypeConditional || np->conditional.type != cudaGraphCondTypeWhile)
        return cudaErrorNotSupported;
    auto body = std::make_shared<HostGraph>();
    static cudaGraph_t out[1];
    out[0] = body.get();
    np->conditional.phGraph_out = out;
    unsigned* v = reinterpret_cast<unsigned*>(np->conditional.handle);
    g->ops.push_back([v, body]() {
        while (*v)
            for (auto& f : body->ops) f();
    });
    *node = nullptr;
    return cudaSuccess;
}
inline cudaError_t cudaStreamUpdateCaptureDependencies(cudaStream_t, cudaGraphNode_t*, const cudaGraphEdgeData*,
                                                       size_t, unsigned) {
    return cudaSuccess;
}
inline cudaError_t cudaStreamBeginCaptureToGraph(cudaStream_t, cudaGraph_t g, const cudaGraphNode_t*,
                                                 const cudaGraphEdgeData*, size_t, cudaStreamCaptureMode) {
    host_captures().push_back(g);
    return cudaSuccess;
}
inline cudaError_t cudaGraphInstantiate(cudaGraphExec_t* e, cudaGraph_t g, unsigned long long) {
    *e = new HostGraph(*g);
    return cudaSuccess;
}
inline cudaError_t cudaGraphLaunch(cudaGraphExec_t e, cudaStream_t) {
    for (auto& f : e->ops) f();
    return cudaSuccess;
}
inline cudaError_t cudaGraphDestroy(cudaGraph_t g) { delete g; return cudaSuccess; }
inline cudaError_t cudaGraphExecDestroy(cudaGraphExec_t e) { delete e; return cudaSuccess; }
inline cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned) {
    static int dummy;
    *s = &dummy;
    return cudaSuccess;
}
inline cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }

inline cudaError_t cudaMemsetAsync(void* p, int v, size_t n, cudaStream_t = nullptr) {
    return host_submit([=]() { std::memset(p, v, n); return cudaSuccess; });
}
inline cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind,
                                   cudaStream_t = nullptr) {
    return host_submit([=]() { std::memcpy(d, s, n); return cudaSuccess; });
}
inline cudaError_t cudaMemcpy(void* d, const void* s, size_t n, cudaMemcpyKind) {
    std::memcpy(d, s, n);
    return cudaSuccess;
}
inline cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
typedef struct CUevent_st* cudaEvent_t;
inline cudaError_t cudaEventCreate(cudaEvent_t* e) { *e = nullptr; return cudaSuccess; }
inline cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
inline cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t = nullptr) { return cudaSuccess; }
inline cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned) { *e = nullptr; return cudaSuccess; }
inline cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned) { return cudaSuccess; }
inline cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t, cudaEvent_t) { *ms = 0.f; return cudaSuccess; }
inline cudaError_t cudaGetLastError() { return cudaSuccess; }
inline cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
enum cudaDeviceAttr { cudaDevAttrMultiProcessorCount = 16 };
inline cudaError_t cudaGetDevice(int*) { return cudaErrorNotSupported; }  // no device: keep the default
inline cudaError_t cudaDeviceGetAttribute(int*, cudaDeviceAttr, int) { return cudaErrorNotSupported; }
inline const char* cudaGetErrorString(cudaError_t) { return "host test double error"; }
