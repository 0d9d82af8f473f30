// AAb_Solver kernels for quantised storage of SA (bf16, and fp8 e4m3 with one
// scale per 128 × 128 tile); the arithmetic stays fp32 (the sketch only
// preconditions the iteration, Section 3.1).  Instantiated here, apart from
// the fp32 kernels, so that the translation units compile in parallel.
#include "aab_kernel.cuh"

namespace mihs {
namespace aabk {

AabKernelFn kernel_for_bf16(int cl, int dp) { return kernel_for_type<__nv_bfloat16>(cl, dp); }
AabKernelFn kernel_for_fp8(int cl, int dp) { return kernel_for_type<__nv_fp8_e4m3>(cl, dp); }

}  // namespace aabk
}  // namespace mihs
