// Tensor-core V-list M2L for the MIXED path (tcgen05, split-bf16 products).
#include "internal.h"

namespace pk {

void m2l_tc_prepare(Plan &) {}
bool m2l_tc_run(Plan &, cudaStream_t) { return false; }

}  // namespace pk
