// One CUDA graph for a whole CTMRG convergence (see graph.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace ipeps {

// Builds a graph from the work a host routine issues on one stream.  Straight-line work is stream
// captured (cudaStreamBeginCaptureToGraph) segment by segment; a loop becomes a conditional WHILE
// node whose body is captured the same way, so loops nest.  The loop's condition is set on the
// device: loop_begin launches an arming kernel (condition 1, counter 0) ahead of the node, and the
// body's last test kernel sets it to continue or stop.  Capture mode is thread-local, so other host
// threads driving other handles are not affected.
class GraphBuilder {
 public:
  ~GraphBuilder();
  int begin(cudaStream_t st);
  // arms and opens a WHILE loop; *h_out is the condition handle for the body's test kernel;
  // *ctr is zeroed by the arming kernel (the body's test kernel counts rounds in it)
  int loop_begin(int* ctr, cudaGraphConditionalHandle* h_out);
  int loop_end();
  // closes the outer capture and instantiates the graph
  int end(cudaGraphExec_t* exec_out);
  // ends a capture left open by an error and drops the graph
  void abandon();
  bool active() const { return !stack_.empty(); }

 private:
  struct Level {
    cudaGraph_t g;
    std::vector<cudaGraphNode_t> deps;
  };
  int seg_begin();
  int seg_end();
  std::vector<Level> stack_;
  cudaGraph_t root_ = nullptr;
  cudaStream_t st_ = nullptr;
  bool capturing_ = false;
};

// Device side of a loop: *ctr = 0 and (graph mode) condition = 1.  In eager mode (graph = 0) the
// same kernel only resets the counter, so both modes run the same kernels.
__global__ void loop_arm_kernel(cudaGraphConditionalHandle h, int graph, int* ctr);

__device__ __forceinline__ void loop_set(cudaGraphConditionalHandle h, int graph, bool cont) {
  if (graph) cudaGraphSetConditional(h, cont ? 1u : 0u);
}

}  // namespace ipeps
