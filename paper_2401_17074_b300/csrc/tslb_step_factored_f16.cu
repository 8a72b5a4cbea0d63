// The factored step instantiated for CodecF16 and CodecF16SR storage (kernels in tslb_step_factored.cuh).
#include "tslb_step_factored.cuh"

namespace tslb {

cudaError_t launch_factored_CodecF16(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo, int zhi) {
    return launch_codec<CodecF16>(h, src, dst, p, zlo, zhi);
}

cudaError_t launch_factored_CodecF16SR(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo, int zhi) {
    return launch_codec<CodecF16SR>(h, src, dst, p, zlo, zhi);
}

}  // namespace tslb
