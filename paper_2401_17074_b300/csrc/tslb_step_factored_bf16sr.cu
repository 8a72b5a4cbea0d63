// The factored step instantiated for CodecBF16SR storage (kernels in tslb_step_factored.cuh; one
// storage type per translation unit: the compiles run in parallel, and each instance is
// compiled on its own, which gave the 16-bit kernels fewer spills than a shared unit).
#include "tslb_step_factored.cuh"

namespace tslb {

cudaError_t launch_factored_CodecBF16SR(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo,
                                 int zhi) {
    return launch_codec<CodecBF16SR>(h, src, dst, p, zlo, zhi);
}

}  // namespace tslb
