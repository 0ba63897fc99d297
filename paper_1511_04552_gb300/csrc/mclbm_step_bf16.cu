// Step kernels of libmclbm for state storage type __nv_bfloat16 (one translation unit per storage
// type, so the build compiles them in parallel).
#include "mclbm_pair.cuh"

namespace mcl {

cudaError_t launch_step_bf16(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                           cudaStream_t st) {
  return pair::launch_pair_t<__nv_bfloat16>(a, c, map, st);
}

cudaError_t prepare_tma_bf16(StepConfig* c, const Layout& L) {
  return pair::prepare_pair_tma_t<__nv_bfloat16>(c, L);
}

}  // namespace mcl
