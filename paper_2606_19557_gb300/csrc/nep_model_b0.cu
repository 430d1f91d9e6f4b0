// Per-atom kernels instantiated for the shape bucket (N_R, K_R, N_A, K_A) <= (5, 9, 5, 9).
#include "nep_model.cuh"

namespace nep {
KernelSet make_bucket0() { return make_set<5, 9, 5, 9>(); }
}  // namespace nep

namespace nep {
KernelSet make_bucket1();
KernelSet make_bucket2();

// Smallest bucket that holds the model sizes (unused channels are zero-padded).
const KernelSet *select_kernels(int nR, int kR, int nA, int kA) {
    static const KernelSet sets[3] = {make_bucket0(), make_bucket1(), make_bucket2()};
    for (const KernelSet &k : sets)
        if (nR <= k.NR && kR <= k.KR && nA <= k.NA && kA <= k.KA) return &k;
    return nullptr;
}
}  // namespace nep
