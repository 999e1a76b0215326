// hg_sc_bf16.cu -- stream-collide instantiations for BF16 storage (see hg_device.cuh).
#include "hg_device.cuh"

namespace hg {

cudaError_t launch_sc_bf16(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles, int64_t n_tiles,
                          int off, int parity, const OneDomain &one, cudaStream_t st) {
    return launch_sc_storage<kBF16>(cfg, doms, tiles, n_tiles, off, parity, one, st);
}

}  // namespace hg
