// hz_krylov_f32.cu -- FP32 instantiation of the inner iteration (mixed-precision solver).
#include "hz_krylov.cuh"

namespace hz {
#define HZ_T float
#include "hz_krylov_inst.inc"
#undef HZ_T
}  // namespace hz
