// Advance-kernel instantiations for 128-thread blocks (one translation unit per block
// size so that nvcc compiles them in parallel).
#include "lpm_advance.cuh"

namespace lpm {
LPM_ADVANCE_TU(128)
}  // namespace lpm
