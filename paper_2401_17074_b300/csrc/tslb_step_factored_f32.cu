// The factored step instantiated for CodecF32 storage (kernels in tslb_step_factored.cuh).
#include "tslb_step_factored.cuh"

namespace tslb {

cudaError_t launch_factored_CodecF32(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo, int zhi) {
    return launch_codec<CodecF32>(h, src, dst, p, zlo, zhi);
}

}  // namespace tslb
