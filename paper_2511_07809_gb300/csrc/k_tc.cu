// BF16 tensor-core (tcgen05 / TMEM) form of the CP-step contractions.
#include "tlda_internal.h"

namespace tlda {
void launch_qy_tc(const StepArgs &, cudaStream_t) {}
void launch_zh_tc(const StepArgs &, cudaStream_t) {}
void launch_g_tc(const StepArgs &, cudaStream_t) {}
}  // namespace tlda
