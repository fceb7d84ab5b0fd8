// hz_krylov_f64.cu -- FP64 instantiation of the inner iteration (double-precision solver).
#include "hz_krylov.cuh"

namespace hz {
#define HZ_T double
#include "hz_krylov_inst.inc"
#undef HZ_T
}  // namespace hz
