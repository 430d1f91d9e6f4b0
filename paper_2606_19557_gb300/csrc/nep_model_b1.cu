// Per-atom kernels instantiated for the shape bucket (N_R, K_R, N_A, K_A) <= (7, 11, 7, 11).
#include "nep_model.cuh"

namespace nep {
KernelSet make_bucket1() { return make_set<7, 11, 7, 11>(); }
}  // namespace nep
