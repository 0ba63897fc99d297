// Step kernels of libmclbm for state storage type __nv_bfloat16 (one translation unit per storage
// type, so the build compiles them in parallel).
#include "mclbm_pair.cuh"

namespace mcl {

cudaError_t launch_step_bf16(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                           cudaStream_t st) {
  if (c.variant >= 10) {  // the one-node-per-thread kernels (comparisons)
    StepConfig c1 = c;
    c1.variant -= 10;
    return launch_step_t<__nv_bfloat16>(a, c1, map, st);
  }
  return pair::launch_pair_t<__nv_bfloat16>(a, c, map, st);
}

cudaError_t prepare_tma_bf16(StepConfig* c, const Layout& L) {
  return c->variant >= 10 ? prepare_tma_t<__nv_bfloat16>(c, L) : pair::prepare_pair_tma_t<__nv_bfloat16>(c, L);
}

}  // namespace mcl
