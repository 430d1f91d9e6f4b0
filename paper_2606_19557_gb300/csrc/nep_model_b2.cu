// Per-atom kernels instantiated for the shape bucket (N_R, K_R, N_A, K_A) <= (12, 12, 12, 12).
#include "nep_model.cuh"

namespace nep {
KernelSet make_bucket2() { return make_set<12, 12, 12, 12>(); }
}  // namespace nep
