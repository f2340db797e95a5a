// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) network path.
#include "dpa1.h"
#include "model.h"

namespace dpa1 {

int tc_init_weights(dp_model* m, const HostArrays& arrays, std::string& msg) {
  (void)m; (void)arrays;
  msg = "the BF16 tensor-core path is not available in this build";
  return DP_ERR_UNSUPPORTED;
}
void tc_plan_buffers(dp_model*, Arena&, int) {}
void tc_run_network(dp_model*, int, const int*, cudaStream_t) {}
void tc_free_weights(dp_model* m) {
  for (void* p : m->tcw.allocations) cudaFree(p);
  m->tcw.allocations.clear();
}

}  // namespace dpa1
