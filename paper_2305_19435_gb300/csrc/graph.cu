// Search plans: a fixed-shape AdANNS-IVF search captured once into a CUDA
// graph and replayed with a single launch (no per-call host work besides
// cudaGraphLaunch).  The captured work is the same launch sequence
// adanns_search_ivf issues; scratch comes from graph-owned memory nodes.
#include <vector>

#include "internal.cuh"

struct adanns_plan {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  int kernels = 0;  // kernel nodes in the graph
};

namespace {
void destroy(adanns_plan *p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) cudaStreamDestroy(p->cap);
  delete p;
}
}  // namespace

using namespace adn;

extern "C" {

int adanns_plan_create(const adanns_index *idx, const float *queries, int64_t B, int d_c, int d_s,
                       int nprobe, int k, int storage, int rerank_k, int64_t *out_ids,
                       float *out_dist, void *cuda_stream, adanns_plan **out) {
  if (!out) return fail(ADANNS_ERR_ARG, "out is NULL");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // one ordinary call first: validates the arguments, sets kernel attributes
  // and grows the scratch pool outside the capture
  int rc = adanns_search_ivf(idx, queries, B, d_c, d_s, nprobe, k, storage, rerank_k, out_ids,
                             out_dist, nullptr, cuda_stream);
  if (rc) return rc;
  ADN_CUDA(cudaStreamSynchronize(st));
  adanns_plan *p = new adanns_plan();
  cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "plan stream");
  }
  e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "begin capture");
  }
  rc = adanns_search_ivf(idx, queries, B, d_c, d_s, nprobe, k, storage, rerank_k, out_ids,
                         out_dist, nullptr, p->cap);
  e = cudaStreamEndCapture(p->cap, &p->graph);
  if (rc) {
    destroy(p);
    return rc;
  }
  if (e != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "end capture");
  }
  size_t nn = 0;
  if (cudaGraphGetNodes(p->graph, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(p->graph, nodes.data(), &nn) == cudaSuccess)
      for (auto n : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++p->kernels;
      }
  }
  cudaGetLastError();
  e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (e != cudaSuccess) {
    destroy(p);
    return cuda_fail(e, "instantiate");
  }
  *out = p;
  return ADANNS_OK;
}

int adanns_plan_launch(adanns_plan *plan, void *cuda_stream) {
  if (!plan || !plan->exec) return fail(ADANNS_ERR_ARG, "plan is NULL");
  ADN_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)cuda_stream));
  g_launches.fetch_add(plan->kernels, std::memory_order_relaxed);
  return ADANNS_OK;
}

void adanns_plan_free(adanns_plan *plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  destroy(plan);
}

}  // extern "C"
