// Filter kernels of htex_lookup for e4m3 texels (one translation unit
// per texel format, compiled in parallel).
#include "lookup_kernels.cuh"

namespace htex {

htex_status launch_fwd_e4m3(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s, bool binned) {
    return binned ? launch_fwd_c<HTEX_E4M3, true>(t, p, flags, s) : launch_fwd_c<HTEX_E4M3, false>(t, p, flags, s);
}

}  // namespace htex
