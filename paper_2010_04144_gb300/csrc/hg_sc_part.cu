// hg_sc_part.cu -- the stream-collide kernels of one (storage, scheme, launch parity)
// combination, given by HG_PART_S, HG_PART_SCHEME and HG_PART_PAR at compile time
// (see launch_sc_part in hg_internal.h).  The build compiles this file once per
// combination, so the twelve sets of instantiations compile in parallel.
#include "hg_device.cuh"

#if !defined(HG_PART_S) || !defined(HG_PART_SCHEME) || !defined(HG_PART_PAR)
#error "compile with -DHG_PART_S=.. -DHG_PART_SCHEME=.. -DHG_PART_PAR=.."
#endif

namespace hg {

template <>
cudaError_t launch_sc_part<HG_PART_S, HG_PART_SCHEME, HG_PART_PAR>(const CollideCfg &cfg, const DomDev *doms,
                                                                   const TileDev *tiles, int64_t n_tiles, int off,
                                                                   const OneDomain &one, cudaStream_t st) {
    return launch_sc_spt<HG_PART_S, HG_PART_SCHEME, HG_PART_PAR>(cfg, doms, tiles, n_tiles, off, one, st);
}

}  // namespace hg
