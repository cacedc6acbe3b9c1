// Graph builder for device-driven loops (graph.cuh).
//
// The CTMRG convergence loop and the projector's subspace-round loop both end on conditions the
// device computes (every instance frozen; every subspace problem accepted).  Issued eagerly they
// need a host readback to decide whether to continue; as conditional WHILE nodes of one graph the
// device decides and the host sees one graph launch per convergence.
#include "common.cuh"
#include "graph.cuh"

namespace ipeps {

__global__ void loop_arm_kernel(cudaGraphConditionalHandle h, int graph, int* ctr) {
  if (threadIdx.x == 0) {
    *ctr = 0;
    loop_set(h, graph, true);
  }
}

GraphBuilder::~GraphBuilder() { abandon(); }

int GraphBuilder::seg_begin() {
  Level& L = stack_.back();
  IPEPS_CUDA_TRY(cudaStreamBeginCaptureToGraph(st_, L.g, L.deps.empty() ? nullptr : L.deps.data(), nullptr,
                                               L.deps.size(), cudaStreamCaptureModeThreadLocal));
  capturing_ = true;
  return 0;
}

int GraphBuilder::seg_end() {
  Level& L = stack_.back();
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* deps = nullptr;
  size_t n = 0;
  IPEPS_CUDA_TRY(cudaStreamGetCaptureInfo(st_, &status, nullptr, nullptr, &deps, nullptr, &n));
  if (status != cudaStreamCaptureStatusActive)
    return cuda_fail(cudaErrorStreamCaptureInvalidated, "graph capture invalidated", __FILE__, __LINE__);
  L.deps.assign(deps, deps + n);
  cudaGraph_t out = nullptr;
  capturing_ = false;
  IPEPS_CUDA_TRY(cudaStreamEndCapture(st_, &out));
  return 0;
}

int GraphBuilder::begin(cudaStream_t st) {
  abandon();
  st_ = st;
  IPEPS_CUDA_TRY(cudaGraphCreate(&root_, 0));
  stack_.push_back(Level{root_, {}});
  return seg_begin();
}

int GraphBuilder::loop_begin(int* ctr, cudaGraphConditionalHandle* h_out) {
  Level& L = stack_.back();
  cudaGraphConditionalHandle h;
  IPEPS_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, L.g, 0, 0));
  loop_arm_kernel<<<1, 32, 0, st_>>>(h, 1, ctr);
  IPEPS_CUDA_TRY(cudaGetLastError());
  if (int rc = seg_end()) return rc;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  IPEPS_CUDA_TRY(cudaGraphAddNode(&node, L.g, L.deps.empty() ? nullptr : L.deps.data(), nullptr, L.deps.size(), &p));
  L.deps.assign(1, node);
  stack_.push_back(Level{p.conditional.phGraph_out[0], {}});
  *h_out = h;
  return seg_begin();
}

int GraphBuilder::loop_end() {
  if (stack_.size() < 2) return cuda_fail(cudaErrorInvalidValue, "graph loop_end without loop", __FILE__, __LINE__);
  if (int rc = seg_end()) return rc;
  stack_.pop_back();
  return seg_begin();
}

int GraphBuilder::end(cudaGraphExec_t* exec_out) {
  if (stack_.size() != 1) return cuda_fail(cudaErrorInvalidValue, "graph end inside a loop", __FILE__, __LINE__);
  if (int rc = seg_end()) return rc;
  stack_.clear();
  cudaError_t e = cudaGraphInstantiate(exec_out, root_, 0);
  cudaGraphDestroy(root_);
  root_ = nullptr;
  IPEPS_CUDA_TRY(e);
  return 0;
}

void GraphBuilder::abandon() {
  if (capturing_) {
    cudaGraph_t out = nullptr;
    cudaStreamEndCapture(st_, &out);
    cudaGetLastError();
    capturing_ = false;
  }
  stack_.clear();
  if (root_) cudaGraphDestroy(root_);
  root_ = nullptr;
}

}  // namespace ipeps
