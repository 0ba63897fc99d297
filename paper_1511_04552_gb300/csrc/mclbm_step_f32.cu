// Step kernels of libmclbm for state storage type float (one translation unit per storage
// type, so the build compiles them in parallel).
#include "mclbm_pair.cuh"
#include "mclbm_pair2.cuh"

namespace mcl {

cudaError_t launch_step_f32(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                           cudaStream_t st) {
  return pair::launch_pair_t<float>(a, c, map, st);
}

cudaError_t prepare_tma_f32(StepConfig* c, const Layout& L) {
  return pair::prepare_pair_tma_t<float>(c, L);
}

cudaError_t prepare_two_f32(StepConfig* c, const Layout& L) { return pair::prepare_two(c, L); }

cudaError_t launch_two_f32(const StepArgs& a, const StepConfig& c, const CUtensorMap* map2,
                           cudaStream_t st) {
  return pair::launch_two(a, c, map2, st);
}

}  // namespace mcl
