// BF16 tensor-core (tcgen05 / TMEM) form of the CP-step contractions.
#include "tlda_internal.h"

namespace tlda {
void launch_chain_bf16(const StepArgs &, cudaStream_t) {}
}  // namespace tlda
